"""Pins of the oracle's minimal-surface residual (Sec. 3, "Minimal Surface")
against facts fixed outside it: F is the gradient of the discrete area, affine
states are exact minimal surfaces, the small-slope limit is the Laplacian, the
assembled Jacobian is the brute-force derivative and symmetric, and the
discrete solution converges at O(h^2) to Scherk's surface, an exact minimal
surface."""
import numpy as np
import pytest

from oracle import adjoint, fem, jfnk
from workloads import random_direction, random_state_field


def _coords(n):
    return fem.node_coords(n, 2)


def test_residual_is_gradient_of_discrete_area():
    n = 6
    u = fem.minsurf_boundary(n) + random_state_field(n, 2, seed=3, kind="uniform", amplitude=0.7)
    F = fem.residual("minsurf2d", u)
    h = 1e-6
    for idx in [(1, 1), (2, 4), (5, 3), (3, 3)]:
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        g = (fem.minsurf_energy(up) - fem.minsurf_energy(um)) / (2 * h)
        assert F[idx] == pytest.approx(g, rel=1e-7, abs=1e-10)
    assert np.all(F[fem.boundary_mask(u.shape)] == 0.0)


def test_affine_states_are_exact_minimal_surfaces():
    n = 9
    x, y = _coords(n)
    u = 0.7 * x - 1.3 * y + 0.2
    F = fem.residual("minsurf2d", u)
    assert np.max(np.abs(F)) <= 1e-14


def test_small_slope_limit_is_the_laplacian():
    """F(delta w) = delta K w + O(delta^3) with K the Q1 stiffness (the Bratu
    residual at lambda = 0)."""
    n = 8
    w = random_state_field(n, 2, seed=5, kind="uniform", amplitude=1.0)
    Kw = fem.residual("bratu2d", w, 0.0)
    errs = []
    for d in (1e-2, 1e-3):
        errs.append(np.linalg.norm(fem.residual("minsurf2d", d * w) / d - Kw) / np.linalg.norm(Kw))
    assert errs[1] <= 1e-3
    assert errs[0] / errs[1] == pytest.approx(100.0, rel=0.05)  # O(delta^2)


def test_jacobian_matches_brute_force_and_is_symmetric():
    n = 5
    u = fem.minsurf_boundary(n) + random_state_field(n, 2, seed=7, kind="uniform", amplitude=0.8)
    J = fem.assemble_jacobian("minsurf2d", u).toarray()
    m = fem.interior(u.shape).ravel()
    h = 1e-6
    cols = []
    for j in np.flatnonzero(m):
        up, um = u.ravel().copy(), u.ravel().copy()
        up[j] += h
        um[j] -= h
        cols.append((fem.residual("minsurf2d", up.reshape(u.shape)) -
                     fem.residual("minsurf2d", um.reshape(u.shape))).ravel() / (2 * h))
    Jfd = np.stack(cols, axis=1)[m]
    Ji = J[m][:, m]
    assert np.max(np.abs(Ji - Jfd)) <= 1e-7 * np.max(np.abs(Ji))
    assert np.allclose(Ji, Ji.T, atol=1e-15)
    assert np.linalg.eigvalsh(Ji).min() > 0.0  # the area is convex


def _scherk(n, a=2.0):
    """Scherk's surface u = (1/a) ln(cos(a(y - 1/2)) / cos(a(x - 1/2))), scaled and
    shifted onto the unit square (a homothety of z = ln(cos y / cos x))."""
    x, y = _coords(n)
    return np.log(np.cos(a * (y - 0.5)) / np.cos(a * (x - 0.5))) / a


def test_discrete_solution_converges_to_scherk_surface():
    errs = []
    for n in (8, 16, 32):
        ue = _scherk(n)
        u0 = ue.copy()
        u0[fem.interior(u0.shape)] = 0.0
        ud, hist = adjoint.newton_direct("minsurf2d", u0)
        assert hist[-1] <= 1e-12 * hist[0]
        errs.append(np.max(np.abs(ud - ue)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= r <= 2.3 for r in rates), (errs, rates)


@pytest.mark.parametrize("opts", ["default", "paper"])
def test_jfnk_mg_solve_matches_exact_newton(opts):
    """The oracle's JFNK-MG solve of the Sec. 3 minimal-surface problem reaches
    the exact-Newton discrete solution."""
    n, levels = 32, 3
    u0 = fem.minsurf_boundary(n)
    lvs = jfnk.build_hierarchy("minsurf2d", n, levels)
    if opts == "paper":
        o = jfnk.paper_options(atol_newton=1e-12)
    else:
        o = jfnk.Options(rtol_newton=1e-11)
    u, st = jfnk.newton_solve(lvs, u0, o)
    assert st.converged
    # undamped exact Newton diverges from u0 on this problem (steep boundary
    # layers); started near the minimiser (unique: the area is convex) it
    # converges quadratically to the discrete solution
    start = u + np.where(fem.interior(u.shape), 1e-3 * random_direction(n, 2, seed=13), 0.0)
    ud, hist = adjoint.newton_direct("minsurf2d", start)
    assert hist[-1] <= 1e-12 * hist[0]
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    # boundary data untouched
    b = fem.boundary_mask(u.shape)
    assert np.array_equal(u[b], u0[b])


def test_fd_action_matches_assembled_jacobian():
    n = 12
    u = fem.minsurf_boundary(n) + random_state_field(n, 2, seed=11, kind="uniform", amplitude=0.5)
    lv = jfnk.Level("minsurf2d", n, 0.0, None, None)
    v = random_direction(n, 2, seed=12)
    Jv = jfnk.fd_jv(lv, u, lv.F(u), v)
    Jex = (fem.assemble_jacobian("minsurf2d", u) @ v.ravel()).reshape(u.shape)
    assert np.linalg.norm(Jv - Jex) <= 1e-6 * np.linalg.norm(Jex)
