"""Pins of the oracle's Neo-Hookean beam (Sec. 3, "Hyperelasticity") against
facts fixed outside it: F is the gradient of the discrete energy, the reference
and rigid rotations are stress free, a uniaxial stretch gives the closed-form
face tractions, the small-strain limit is isotropic linear elasticity (coded
independently), the transfers are adjoint and preserve linear fields, and the
paper's solver reaches an exact-Newton solution, running its spectral shift on
this non-convex problem."""
import numpy as np
import pytest

from golden import paper_tables
from oracle import hyper, jfnk


def _random_state(m, seed, amp=0.02):
    u = hyper.boundary_state(m)
    rng = np.random.default_rng(seed)
    mask = hyper.unknown_mask(u.shape)
    u[mask] += amp * rng.uniform(-1.0, 1.0, size=int(mask.sum()))
    return u


def test_residual_is_gradient_of_discrete_energy():
    m = 1
    u = _random_state(m, 1)
    F = hyper.residual(u)
    h = 1e-6
    for idx in [(0, 0, 3, 0), (1, 0, 5, 1), (1, 1, 9, 2), (0, 1, 1, 1)]:
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        g = (hyper.energy(up) - hyper.energy(um)) / (2 * h)
        assert F[idx] == pytest.approx(g, rel=1e-6, abs=1e-9)
    assert np.all(F[hyper.dirichlet_mask(u.shape)] == 0.0)


def test_reference_and_rigid_rotations_are_stress_free():
    m = 2
    assert np.max(np.abs(hyper.residual(np.zeros(hyper.shape_of(m))))) == 0.0
    x, y, z = hyper.node_coords(m)
    X = np.stack([x, y, z], axis=-1)
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    th = 0.9
    R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K  # Rodrigues
    u = X @ R.T - X + np.array([0.1, -0.2, 0.3])
    assert np.max(np.abs(hyper.residual(u))) <= 1e-13


def test_uniaxial_stretch_face_tractions():
    """u = (alpha - 1) x e_x: P constant, so interior nodes carry no force and a
    node of the free face y = 0 carries -P e_y times its tributary area:
    (0, -lam ln(alpha) h^2, 0) inside the face, half of it on the edge z = 0."""
    m, alpha = 2, 1.3
    h = 1.0 / m
    x, y, z = hyper.node_coords(m)
    u = np.zeros(hyper.shape_of(m))
    u[..., 0] = (alpha - 1.0) * x
    F = hyper.residual(u)
    t = hyper.LAMBDA * np.log(alpha) * h * h
    assert np.max(np.abs(F[1:-1, 1:-1, 1:-1, :])) <= 1e-13
    assert np.allclose(F[1, 0, 5, :], [0.0, -t, 0.0], atol=1e-13)       # face y = 0 (z = 1/2)
    assert np.allclose(F[0, 0, 5, :], [0.0, -t / 2, -t / 2], atol=1e-13)  # edge y = z = 0


def test_small_strain_limit_is_linear_elasticity():
    m = 2
    rng = np.random.default_rng(3)
    w = rng.normal(size=hyper.shape_of(m))
    Kw = hyper.linear_elastic_residual(w)
    errs = [np.linalg.norm(hyper.residual(d * w) / d - Kw) / np.linalg.norm(Kw) for d in (1e-4, 1e-5)]
    assert errs[1] <= 1e-4
    assert errs[0] / errs[1] == pytest.approx(10.0, rel=0.1)  # O(delta)


def _fd_jacobian(u):
    mask = hyper.unknown_mask(u.shape)
    idx = np.flatnonzero(mask)
    J = np.zeros((idx.size, idx.size))
    h = 1e-6
    for j, k in enumerate(idx):
        up, um = u.ravel().copy(), u.ravel().copy()
        up[k] += h
        um[k] -= h
        J[:, j] = (hyper.residual(up.reshape(u.shape)) - hyper.residual(um.reshape(u.shape))).ravel()[idx] / (2 * h)
    return J, idx


def test_jacobian_is_symmetric():
    J, _ = _fd_jacobian(_random_state(1, 4, amp=0.05))
    assert np.max(np.abs(J - J.T)) <= 1e-6 * np.max(np.abs(J))


def test_transfers_adjoint_and_linear_reproduction():
    mc = 1
    rng = np.random.default_rng(5)
    r = rng.normal(size=hyper.shape_of(2 * mc))
    c = rng.normal(size=hyper.shape_of(mc))
    mf, mcm = hyper.unknown_mask(r.shape), hyper.unknown_mask(c.shape)
    lhs = np.sum(hyper.restrict(r) * np.where(mcm, c, 0.0))
    rhs = np.sum(np.where(mf, r, 0.0) * hyper.prolong(c))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # I is the coarse trilinear interpolant at the fine nodes (scipy's
    # interpolator as the independent evaluation), for a correction that
    # vanishes on the Dirichlet faces
    from scipy.interpolate import RegularGridInterpolator
    c = np.where(mcm, c, 0.0)
    h = 1.0 / mc
    axes = (np.arange(mc + 1) * h, np.arange(mc + 1) * h, np.arange(hyper.LENGTH * mc + 1) * h)
    xf, yf, zf = hyper.node_coords(2 * mc)
    pts = np.stack([zf.ravel(), yf.ravel(), xf.ravel()], axis=-1)
    ref = np.stack([RegularGridInterpolator(axes, c[..., k])(pts).reshape(xf.shape) for k in range(3)], -1)
    assert np.allclose(hyper.prolong(c)[mf], ref[mf], atol=1e-13)
    # the projection keeps constants everywhere (the free faces included)
    pc = hyper.project(np.ones(r.shape))
    assert np.allclose(pc, 1.0, atol=1e-15)


def _exact_newton(u, iters=6):
    for _ in range(iters):
        J, idx = _fd_jacobian(u)
        F = hyper.residual(u).ravel()[idx]
        if np.linalg.norm(F) < 1e-13:
            break
        uf = u.ravel().copy()
        uf[idx] -= np.linalg.solve(J, F)
        u = uf.reshape(u.shape)
    return u


def test_paper_solver_on_the_beam():
    """Refinement level L1 (20 x 2 x 2 elements, two levels): the paper's
    solver converges to the solution that exact Newton keeps (to 1e-8), runs
    the spectral shift of Alg. 1 (the beam is non-convex), and needs the
    Newton count of Table 2 to within one step."""
    lvs = jfnk.build_hyper_hierarchy(1)
    u, st = jfnk.newton_solve(lvs, hyper.boundary_state(2), jfnk.paper_options(atol_newton=1e-10))
    assert st.converged
    assert getattr(lvs[0], "shift_calls", 0) > 0
    ue = _exact_newton(u)
    assert np.linalg.norm(u - ue) <= 1e-8 * np.linalg.norm(ue)
    _, st6 = jfnk.newton_solve(jfnk.build_hyper_hierarchy(1), hyper.boundary_state(2), jfnk.paper_options())
    assert abs(st6.newton_its - paper_tables.load()[("table2", "hyper", "newton_its")][0]) <= 1


def test_shifted_coarse_solve_is_discontinuous_at_twisted_states():
    """Where the coarse CG meets negative curvature, the step at which it does
    (and so lambda_c, the shift and the coarse correction) depends on rounding:
    a 1e-13 relative perturbation of the right-hand side moves the V-cycle
    output by O(1).  Iteration counts of the paper's solver on the beam are
    therefore not reproducible across implementations, and V-cycle parity is
    only checked at states where no shift is taken."""
    k, m = 2, 4
    lvs0 = jfnk.build_hyper_hierarchy(k)
    u, _ = jfnk.newton_solve(lvs0, hyper.boundary_state(m), jfnk.paper_options(max_newton=4))
    b = np.where(hyper.unknown_mask(u.shape), np.random.default_rng(10).normal(size=u.shape), 0.0)

    def cycle(rhs):
        lvs = jfnk.build_hyper_hierarchy(k)
        oo = jfnk.paper_options()
        jfnk.setup_levels(lvs, u, oo, 0)
        return jfnk.mg_vcycle(lvs, k, rhs, oo), getattr(lvs[0], "shift_calls", 0)

    s1, sh1 = cycle(b)
    s2, _ = cycle(b * (1.0 + 1e-13 * np.random.default_rng(5).normal(size=b.shape)))
    assert sh1 > 0
    assert np.linalg.norm(s1 - s2) > 1e-3 * np.linalg.norm(s1)
