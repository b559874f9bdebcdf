"""The solve's line search and failure statuses on the GPU, driven from the
host only: the failing input is written into a caller-owned tensor, or comes
from the options, never from a fault on the device.

  * backtracking (Dennis & Schnabel, Sec. 6.3; Sec. 3 "Setup") on a strongly
    nonlinear diffusion problem whose early Newton steps must be cut: the
    accepted steps, trial counts and residual norms against the oracle's;
  * JFNK_ERR_LINESEARCH: one trial allowed where the full step fails; the
    iterate stays the last accepted one;
  * JFNK_ERR_NONFINITE: a NaN written into the initial guess;
  * JFNK_ERR_NOT_CONVERGED: the Newton iteration limit;
  * JFNK_ERR_BREAKDOWN: a preconditioner that returns zero (no smoothing, a
    coarse solve stopped before its first iteration by an absolute tolerance)
    makes the FGMRES least-squares problem singular.
After each failure the same problem solves a regular case, so the status came
back without losing the CUDA context."""
import functools

import numpy as np
import pytest

from gpu_common import dev, host, jf, rel, torch
from oracle import adjoint, jfnk

pytestmark = pytest.mark.gpu

N, LEVELS, C = 16, 3, 1000.0


def _const_load(n, c):
    """Load vector of the constant source f = c: int f phi_i = c h^3 on interior nodes."""
    load = np.zeros((n + 1,) * 3)
    load[1:-1, 1:-1, 1:-1] = c / n ** 3
    return load


def _gpu_nd(**kw):
    o = jf().default_options(nu_pre=2, nu_post=2, cheb_degree=4, **kw)
    return jf().Problem("nd3d", N, LEVELS, load=dev(_const_load(N, C)), options=o)


@functools.lru_cache(maxsize=None)
def _oracle_nd(ls_max):
    lv = jfnk.build_hierarchy("nd3d", N, LEVELS, load=_const_load(N, C))
    o = jfnk.Options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=1e-10, max_newton=30, ls_max=ls_max)
    return jfnk.newton_solve(lv, np.zeros((N + 1,) * 3), o)


def _regular_solve_ok(p):
    u = torch.zeros(p.shape(), dtype=torch.float64, device="cuda")
    st = p.solve(u, check=False)
    return st["status_code"] == 0 and st["converged"]


def test_backtracking_matches_the_oracle():
    p = _gpu_nd(rtol_newton=1e-10, max_newton=30)
    u = torch.zeros(p.shape(), dtype=torch.float64, device="cuda")
    st = p.solve(u)
    uo, so = _oracle_nd(10)
    assert so.converged and st["converged"]
    # the early steps backtrack: some quadratic / cubic steps are clipped to
    # [0.1, 0.5] alpha, the others are interpolation minimisers
    assert so.ls_hist[0] >= 2 and any(0.1 < a < 0.5 for a in so.alpha_hist)
    assert st["newton_its"] == so.newton_its
    assert st["ls_hist"] == so.ls_hist
    # the search directions agree to the FD round-off of the V-cycle (~1e-6
    # relative), and so do the steps chosen from them
    assert np.allclose(st["alpha_hist"], so.alpha_hist, rtol=1e-5, atol=0.0)
    # ||F_k|| agree to ~1e-6 while the steps are damped; once the full steps
    # converge quadratically ||F_(k+1)|| is the linear residual of the last
    # Krylov solve, and the ~1e-6 difference of the directions becomes a
    # larger relative difference of that small remainder (2e-5 at 1e-5 ||F_0||)
    r_gpu, r_ora = np.array(st["res_hist"]), np.array(so.res_hist)
    damped = r_ora > 1e-1 * r_ora[0]
    assert np.allclose(r_gpu[damped], r_ora[damped], rtol=1e-5, atol=0.0)
    big = r_ora > 1e-6 * r_ora[0]
    assert np.allclose(r_gpu[big], r_ora[big], rtol=1e-4, atol=0.0)
    ud, _ = adjoint.newton_direct("nd3d", np.zeros((N + 1,) * 3), load=_const_load(N, C))
    assert rel(host(u), ud) <= 1e-8
    assert rel(uo, ud) <= 1e-8


def test_linesearch_failure_keeps_the_last_accepted_iterate():
    p = _gpu_nd(ls_max=1, max_newton=5)
    u = torch.zeros(p.shape(), dtype=torch.float64, device="cuda")
    st = p.solve(u, check=False)
    uo, so = _oracle_nd(1)
    assert so.status == "linesearch"
    assert jf()._abi.STATUS[st["status_code"]] == "LINESEARCH"
    assert st["newton_its"] == so.newton_its == 1
    assert st["alpha_hist"] == [0.0] and st["ls_hist"] == [1]
    assert st["res_hist"][1] == st["res_hist"][0]
    assert torch.count_nonzero(u).item() == 0
    assert "line search" in jf().last_error()
    assert _regular_solve_ok(_gpu_nd(rtol_newton=1e-8))


def test_nonfinite_initial_guess():
    o = jf().default_options()
    p = jf().Problem("bratu2d", 32, 3, lam=5.0, options=o)
    u = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    u[11, 17] = float("nan")
    st = p.solve(u, check=False)
    assert jf()._abi.STATUS[st["status_code"]] == "NONFINITE"
    assert st["newton_its"] == 0 and not st["converged"]
    assert "non-finite" in jf().last_error()
    assert _regular_solve_ok(p)


def test_newton_iteration_limit():
    o = jf().default_options(max_newton=1, rtol_newton=1e-10)
    p = jf().Problem("bratu2d", 32, 3, lam=5.0, options=o)
    u = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    st = p.solve(u, check=False)
    assert jf()._abi.STATUS[st["status_code"]] == "NOT_CONVERGED"
    assert st["newton_its"] == 1 and st["res_hist"][1] < st["res_hist"][0]
    o2 = jf().default_options(max_newton=20, rtol_newton=1e-10)
    u.zero_()
    assert p.solve(u, options=o2)["converged"]


def test_krylov_breakdown_on_a_zero_preconditioner():
    o = jf().default_options(nu_pre=0, nu_post=0, coarse_tol_mode=1, coarse_tol=1e300)
    p = jf().Problem("bratu2d", 16, 2, lam=5.0, options=o)
    u = torch.zeros((17, 17), dtype=torch.float64, device="cuda")
    st = p.solve(u, check=False)
    assert jf()._abi.STATUS[st["status_code"]] == "BREAKDOWN"
    assert "breakdown" in jf().last_error()
    assert torch.count_nonzero(u).item() == 0
    u.zero_()
    assert p.solve(u, options=jf().default_options())["converged"]
