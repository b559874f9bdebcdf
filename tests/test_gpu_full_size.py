"""Whole solves at the full workload sizes, in the configuration bench.py
times (FP64 129^3, V(2,2) degree 4, FGMRES(30), 1e-8; and 257^3 with the FP32
preconditioner against the all-FP64 solve).  The oracle cannot solve these
sizes in seconds, so it checks what holds at any size:
  * its own element routine evaluates F at sampled nodes of the GPU solution,
    and those entries are at the level the stopping rule allows;
  * the GPU solution is the discrete solution of an O(h^2)-accurate scheme: its
    distance to the manufactured u* falls by ~4 when h halves (65^3 -> 129^3),
    a property of the discrete solution that a wrong operator would break;
  * the FP32-preconditioned and the FP64 solves reach the same discrete
    solution (the preconditioner changes the path, not the answer)."""
import numpy as np
import pytest

from gpu_common import host, jf, rel, torch
from oracle import fem

pytestmark = pytest.mark.gpu


def _solve(n, levels, pc="f64"):
    m = jf()
    o = m.default_options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=1e-8,
                          pc_dtype=m.F32 if pc == "f32" else m.F64,
                          eps_mode_pc=m.EPS_FP32 if pc == "f32" else m.EPS_PAPER,
                          power_iters=30, power_tol=1e-2)  # the power method's Sec. 2 rule
    p = m.Problem("nd3d", n, levels, options=o)
    u = torch.zeros((n + 1,) * 3, dtype=torch.float64, device="cuda")
    st = p.solve(u)
    return host(u), st


def _mms_error(u, n):
    x, y, z = fem.node_coords(n, 3)
    return np.max(np.abs(u - fem.mms_exact(x, y, z)))


def test_bench_workload_solution_properties():
    n = 128
    u, st = _solve(n, 6)
    assert st["converged"] and st["newton_its"] <= 8
    # sampled residual entries by the oracle's element routine
    rng = np.random.default_rng(3)
    nodes = [tuple(rng.integers(1, n, size=3)) for _ in range(40)]
    Fs = fem.residual_at("nd3d", u, nodes) - fem.mms_load_at(n, nodes)
    F0 = fem.mms_load_at(n, nodes)  # F at u0 = 0 is -b
    assert np.max(np.abs(Fs)) <= 1e-6 * np.max(np.abs(F0))
    # O(h^2) against the manufactured solution: 65^3 -> 129^3 divides the error by ~4
    u65, st65 = _solve(64, 5)
    e65, e129 = _mms_error(u65, 64), _mms_error(u, n)
    assert 3.3 <= e65 / e129 <= 4.7, (e65, e129)


def test_257_fp32_preconditioner_reaches_the_fp64_solution():
    n = 256
    u64, st64 = _solve(n, 7)
    u32, st32 = _solve(n, 7, pc="f32")
    assert st64["converged"] and st32["converged"]
    assert rel(u32, u64) <= 1e-8
    u128, _ = _solve(128, 6)
    ratio = _mms_error(u128, 128) / _mms_error(u64, n)
    assert 3.3 <= ratio <= 4.7, ratio
