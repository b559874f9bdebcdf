"""GPU parity of the minimal-surface problem (Sec. 3, "Minimal Surface") against
the oracle through the C ABI: the residual element by element, the FD action,
and whole JFNK-MG solves (the default FGMRES settings and the paper's own
settings) on the paper's Dirichlet data u = x(1-x) on y = 0, 1 and 0 on
x = 0, 1."""
import numpy as np
import pytest

from gpu_common import dev, host, jf, rel, torch
from oracle import adjoint, fem, jfnk
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52


def _state(n, seed, amplitude=0.6):
    return fem.minsurf_boundary(n) + random_state_field(n, 2, seed=seed, kind="uniform", amplitude=amplitude)


@pytest.mark.parametrize("n", [7, 64, 95, 600])
def test_residual_parity(n):
    p = jf().Problem("minsurf2d", n, 1)
    u = _state(n, seed=n)
    F_ora = fem.residual("minsurf2d", u)
    F64 = host(p.residual(dev(u)))
    assert rel(F64, F_ora) <= 1e-12
    assert np.all(F64[fem.boundary_mask(u.shape)] == 0)
    F32 = host(p.residual(dev(u, torch.float32)))
    assert rel(F32, F_ora) <= 1e-5


@pytest.mark.parametrize("n", [64, 95])
def test_jvp_parity(n):
    p = jf().Problem("minsurf2d", n, 1)
    u = _state(n, seed=3)
    v = random_direction(n, 2, seed=4)
    ud = dev(u)
    Jv = host(p.jvp(ud, p.residual(ud), dev(v)))
    lv = jfnk.Level("minsurf2d", n, 0.0, None, None)
    Jo = jfnk.fd_jv(lv, u, lv.F(u), v)
    eps = jfnk.fd_eps(u, v, lv.mask)
    # FD round-off bound c eps_p ||F terms|| / eps (c = 64), as for the other problems
    A_abs = np.abs(fem.residual("bratu2d", np.abs(u), 0.0))
    bound = 64 * EPS64 * np.linalg.norm(A_abs) * 4 / eps / np.linalg.norm(Jo)
    assert rel(Jv, Jo) <= max(bound, 1e-12)
    Jex = (fem.assemble_jacobian("minsurf2d", u) @ v.ravel()).reshape(u.shape)
    assert rel(Jv, Jex) <= 1e-5


@pytest.mark.parametrize("pc", ["f64", "f32"])
def test_solve_matches_oracle_solution(pc):
    n, levels = 64, 4
    m = jf()
    o = m.default_options(rtol_newton=1e-11, pc_dtype=m.F32 if pc == "f32" else m.F64,
                          eps_mode_pc=m.EPS_FP32 if pc == "f32" else m.EPS_PAPER)
    p = m.Problem("minsurf2d", n, levels, options=o)
    u0 = fem.minsurf_boundary(n)
    u = dev(u0)
    st = p.solve(u)
    assert st["converged"]
    lvs = jfnk.build_hierarchy("minsurf2d", n, levels)
    uo, so = jfnk.newton_solve(lvs, u0, jfnk.Options(rtol_newton=1e-11))
    assert so.converged
    assert rel(host(u), uo) <= 1e-8
    b = fem.boundary_mask(u0.shape)
    assert np.array_equal(host(u)[b], u0[b])


@pytest.mark.parametrize("n,levels", [(50, 2), (100, 3)])
def test_paper_variant_solve(n, levels):
    """The paper's settings (CG outer, V(5,5), coarse CG-QN with shift,
    ||F|| < 1e-6) on its minimal-surface grids: converged, and the Newton and
    CG counts and GE of the oracle's run of the same algorithm."""
    p = jf().Problem("minsurf2d", n, levels, options=jf().paper_options())
    u0 = fem.minsurf_boundary(n)
    u = dev(u0)
    st = p.solve(u)
    assert st["converged"]
    lvs = jfnk.build_hierarchy("minsurf2d", n, levels)
    uo, so = jfnk.newton_solve(lvs, u0, jfnk.paper_options())
    assert abs(st["newton_its"] - so.newton_its) <= 1
    assert abs(st["ge"] - so.ge) <= 0.2 * so.ge, (st["ge"], so.ge)
    # both iterates satisfy ||F|| < 1e-6 and so agree to the conditioning of J
    ud, _ = adjoint.newton_direct("minsurf2d", uo)
    assert rel(host(u), ud) <= 1e-4


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_paper_variant_counts_match_the_oracle_at_every_level(k):
    """The paper's solver on the minimal surface at the refinement levels L1..L5
    (25 * 2^k elements, k + 1 levels; Sec. 3): the Newton and CG counts of the
    oracle's run of the same algorithm (stored by
    tests/golden/make_minsurf_counts.py), and its GE to within 3 % (the GPU takes
    A(u) of the finest level in the set-up from the Newton residual, one
    evaluation fewer per Newton step)."""
    from golden import make_minsurf_counts
    newton, cg, ge = make_minsurf_counts.load()[k]
    n = 25 * 2 ** k
    p = jf().Problem("minsurf2d", n, k + 1, options=jf().paper_options())
    u = dev(fem.minsurf_boundary(n))
    st = p.solve(u)
    assert st["converged"]
    assert st["newton_its"] == newton and st["linear_its"] == cg, (st["newton_its"], st["linear_its"], newton, cg)
    assert abs(st["ge"] - ge) <= 0.03 * ge, (st["ge"], ge)
