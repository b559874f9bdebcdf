"""GPU parity of the paper's own solver variant (outer CG, coarse CG with the
L-BFGS preconditioner and the spectral shift of Alg. 1, the settings of
Sec. 3) against the oracle, through the C ABI, on the paper's Bratu grids
(25 elements per direction on the coarsest level, Sec. 3)."""
import numpy as np
import pytest

from gpu_common import dev, host, jf, rel, torch
from oracle import adjoint, fem, jfnk
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu


class _LinearLevel(jfnk.Level):
    """Oracle level with the exact linearisation as F (FD action = exact J v)."""

    def __init__(self, lv):
        super().__init__(lv.kind, lv.n, lv.lam, lv.kappa, lv.load)
        self.x0 = lv.x
        self.J = fem.assemble_jacobian(lv.kind, lv.x, lv.lam, lv.kappa)

    def F(self, w):
        self.ge += 1
        return (self.J @ (w - self.x0).ravel()).reshape(w.shape)


def _pair(n, levels, amplitude=0.5, offset=0.0, lam=5.0):
    o = jf().paper_options()
    p = jf().Problem("bratu2d", n, levels, lam=lam, options=o)
    u = random_state_field(n, 2, seed=9, kind="uniform", amplitude=amplitude)
    u[fem.interior(u.shape)] += offset
    p.mg_setup(dev(u), 0)
    lv = jfnk.build_hierarchy("bratu2d", n, levels, lam=lam)
    oo = jfnk.paper_options()
    jfnk.setup_levels(lv, u, oo, 0)
    return p, o, lv, oo, u


def test_coarse_cgqn_parity_first_and_preconditioned_call():
    """First call: plain CG collecting the secant pairs; second call: CG
    preconditioned by the kept pairs.  Both agree with the oracle to the FD
    accuracy of the configuration (3x the oracle's own FD-vs-exact deviation)."""
    n, levels = 50, 2
    p, o, lv, oo, u = _pair(n, levels)
    lv0 = lv[0]
    ll = _LinearLevel(lv0)
    ll.lbfgs = None
    maxit = lv0.n_unknowns
    for seed in (41, 42):
        b = random_direction(25, 2, seed=seed)
        s = host(p.coarse_solve(dev(b)))
        so, _ = jfnk.coarse_cgqn(lambda v: jfnk.fd_jv(lv0, lv0.x, lv0.Fx, v), b, lv0, oo.coarse_tol, maxit,
                                 oo.lbfgs_pairs, oo.shift_gamma)
        se, _ = jfnk.coarse_cgqn(lambda v: jfnk.fd_jv(ll, lv0.x, np.zeros_like(b), v), b, ll, oo.coarse_tol, maxit,
                                 oo.lbfgs_pairs, oo.shift_gamma)
        tol = max(1e-9, 3.0 * rel(so, se))
        assert rel(s, so) <= tol, (seed, rel(s, so), tol)
        # and s solves the coarse linear system to the CG tolerance
        assert rel((ll.J @ s.ravel()).reshape(s.shape), np.where(lv0.mask, b, 0.0)) <= 1e-6


def test_coarse_cgqn_spectral_shift_on_indefinite_jacobian():
    """At u = 2.5 + noise the Bratu Jacobian K - lambda M e^u is indefinite on
    the 25 x 25 coarse grid: CG meets negative curvature and Alg. 1 re-runs it on
    the shifted operator.  The GPU result solves the same shifted system as
    the oracle's (to FD accuracy)."""
    n, levels = 25, 1
    p, o, lv, oo, u = _pair(n, levels, amplitude=0.2, offset=2.5)
    lv0 = lv[0]
    J = fem.assemble_jacobian("bratu2d", lv0.x, 5.0, None)
    m = lv0.mask.ravel()
    assert np.linalg.eigvalsh(J[m][:, m].toarray()).min() < 0.0
    b = random_direction(n, 2, seed=43)
    s = host(p.coarse_solve(dev(b)))
    so, shifts = jfnk.coarse_cgqn(lambda v: jfnk.fd_jv(lv0, lv0.x, lv0.Fx, v), b, lv0, oo.coarse_tol,
                                  lv0.n_unknowns, oo.lbfgs_pairs, oo.shift_gamma)
    assert len(shifts) >= 2
    As = J[m][:, m].toarray() - shifts[-1] * np.eye(int(m.sum()))
    assert np.linalg.eigvalsh(As).min() > 0.0
    # the GPU solution solves the oracle's final shifted system
    bi = b.ravel()[m]
    assert np.linalg.norm(As @ s.ravel()[m] - bi) <= 1e-5 * np.linalg.norm(bi)
    assert rel(s, so) <= 1e-5


@pytest.mark.parametrize("n,levels", [(50, 2), (100, 3), (200, 4)])
def test_paper_solve_bratu_newton_count_and_ge(n, levels):
    """Bratu lambda = 5, the paper's settings: 3 inexact-Newton iterations at
    every refinement level (Table 2) and the oracle's GE count to within 15 %."""
    o = jf().paper_options()
    p = jf().Problem("bratu2d", n, levels, lam=5.0, options=o)
    u = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
    st = p.solve(u)
    assert st["converged"] and st["newton_its"] == 3
    lvs = jfnk.build_hierarchy("bratu2d", n, levels, lam=5.0)
    _, so = jfnk.newton_solve(lvs, np.zeros((n + 1, n + 1)), jfnk.paper_options())
    assert abs(st["ge"] - so.ge) <= 0.15 * so.ge, (st["ge"], so.ge)
    assert abs(st["linear_its"] - so.linear_its) <= 2


def test_paper_solve_bratu_reaches_exact_newton_solution():
    n, levels = 100, 3
    o = jf().paper_options(atol_newton=1e-12)
    p = jf().Problem("bratu2d", n, levels, lam=5.0, options=o)
    u = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
    st = p.solve(u)
    assert st["converged"]
    ud, _ = adjoint.newton_direct("bratu2d", np.zeros((n + 1, n + 1)), lam=5.0)
    assert rel(host(u), ud) <= 1e-8
    assert st["coarse_shifts"] == 0 and st["outer_negcurv"] == 0
