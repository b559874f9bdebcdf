"""Pins of the oracle's discretisation against facts fixed outside the oracle:
closed forms, the energy whose gradient F is (Sec. 1), brute-force
differentiation, partition of unity and manufactured-solution convergence."""
import numpy as np
import pytest

from oracle import adjoint, fem
from workloads import random_direction, random_state_field


def _eig_1d(n):
    j = np.arange(1, n)
    th = j * np.pi / n
    return np.sin(th / 2) ** 2, 2.0 + np.cos(th)


def _sine_mode(n, d, modes):
    t = np.linspace(0.0, 1.0, n + 1)
    grids = np.meshgrid(*([t] * d), indexing="ij")  # array order (z,y,x) / (y,x)
    v = np.ones((n + 1,) * d)
    for g, m in zip(reversed(grids), modes):  # modes given x first
        v = v * np.sin(m * np.pi * g)
    v[fem.boundary_mask(v.shape)] = 0.0
    return v


def test_bratu_residual_is_energy_gradient():
    """Sec. 1: F = grad Psi.  Central differences of the independently written
    discrete energy reproduce F at every interior node."""
    n, lam = 6, 5.0
    u = random_state_field(n, 2, seed=11, amplitude=0.7)
    F = fem.residual("bratu2d", u, lam)
    t = 1e-5
    G = np.zeros_like(u)
    for idx in zip(*np.nonzero(fem.interior(u.shape))):
        up = u.copy(); up[idx] += t
        um = u.copy(); um[idx] -= t
        G[idx] = (fem.bratu_energy(up, lam) - fem.bratu_energy(um, lam)) / (2 * t)
    assert np.max(np.abs(G - F)) <= 1e-8 * np.max(np.abs(F))


def test_bratu_constant_state_closed_form():
    """u = c everywhere (boundary data c): grad u = 0, so F_i = -lam e^c int phi_i = -lam e^c h^2."""
    n, lam, c = 8, 5.0, 0.3
    u = np.full((n + 1, n + 1), c)
    F = fem.residual("bratu2d", u, lam)
    m = fem.interior(u.shape)
    assert np.allclose(F[m], -lam * np.exp(c) / n ** 2, rtol=1e-14, atol=0)
    assert np.all(F[~m] == 0)


def test_nd_linear_state_closed_form():
    """u = x (exact in Q1): A(u)_i = int (1+x^2) d_x phi_i = -int 2x phi_i = -2 x_i h^3,
    the 2-point rule being exact for this integrand."""
    n = 6
    x, y, z = fem.node_coords(n, 3)
    A = fem.operator("nd3d", x.copy())
    m = fem.interior(x.shape)
    h = 1.0 / n
    assert np.allclose(A[m], -2.0 * x[m] * h ** 3, rtol=1e-12, atol=1e-16)


def test_ndk_unit_load_and_constant_coefficient():
    n = 5
    b = fem.unit_load((n + 1,) * 3)
    m = fem.interior(b.shape)
    assert np.allclose(b[m], (1.0 / n) ** 3, rtol=1e-14)
    u = random_state_field(n, 3, seed=3, kind="uniform", amplitude=0.5)
    kap = np.full((n, n, n), 2.5)
    # kappa enters linearly per element: constant kappa scales the operator
    assert np.allclose(fem.operator("ndk3d", u, kappa=kap), 2.5 * fem.operator("nd3d", u), rtol=1e-13, atol=1e-17)


def test_ndk_single_element_partition_of_unity():
    """kappa = indicator of one interior element: only its 2^d nodes receive
    contributions and they sum to zero (sum_a phi_a = 1 on the element)."""
    n = 5
    u = random_state_field(n, 3, seed=5, amplitude=0.8)
    kap = np.zeros((n, n, n))
    kap[2, 1, 2] = 1.7
    A = fem.operator("ndk3d", u, kappa=kap)
    nz = np.argwhere(A != 0)
    assert len(nz) == 8
    assert abs(A.sum()) <= 1e-15 * np.abs(A).sum()
    assert set(map(tuple, nz)) == {(2 + a, 1 + b, 2 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}


@pytest.mark.parametrize("modes", [(1, 1), (3, 2), (5, 7)])
def test_bratu_linearisation_eigenvalues_closed_form(modes):
    """J(0) = K - lam M for Bratu.  On the sine mode (j,k) its eigenvalue is
    (4/3)(s_j c_k + c_j s_k) - lam h^2 c_j c_k / 9 with s = sin^2(theta/2),
    c = 2 + cos(theta), theta = j pi / n.  Central differences of F at 0."""
    n, lam = 8, 5.0
    v = _sine_mode(n, 2, modes)
    t = 1e-4
    Jv = (fem.residual("bratu2d", t * v, lam) - fem.residual("bratu2d", -t * v, lam)) / (2 * t)
    s, c = _eig_1d(n)
    j, k = modes
    h = 1.0 / n
    mu = (4.0 / 3.0) * (s[j - 1] * c[k - 1] + c[j - 1] * s[k - 1]) - lam * h * h * c[j - 1] * c[k - 1] / 9.0
    assert np.max(np.abs(Jv - mu * v)) <= 1e-7 * abs(mu)


@pytest.mark.parametrize("modes", [(1, 1, 1), (2, 3, 1), (5, 5, 4)])
def test_nd_linear_limit_eigenvalues_closed_form(modes):
    """A is odd and A'(0) = K: (A(t v) - A(-t v)) / 2t -> K v, with eigenvalue
    (4h/9)(s_i c_j c_k + c_i s_j c_k + c_i c_j s_k) on the sine modes."""
    n = 6
    v = _sine_mode(n, 3, modes)
    t = 1e-4
    Kv = (fem.operator("nd3d", t * v) - fem.operator("nd3d", -t * v)) / (2 * t)
    s, c = _eig_1d(n)
    i, j, k = [m - 1 for m in modes]
    h = 1.0 / n
    mu = 4 * h / 9 * (s[i] * c[j] * c[k] + c[i] * s[j] * c[k] + c[i] * c[j] * s[k])
    assert np.max(np.abs(Kv - mu * v)) <= 1e-7 * mu


@pytest.mark.parametrize("kind,n", [("bratu2d", 4), ("nd3d", 3), ("ndk3d", 3)])
def test_assembled_jacobian_matches_brute_force(kind, n):
    """The assembled analytic J equals the dense Jacobian built column by column
    from central differences of F."""
    d = fem.dim_of(kind)
    u = random_state_field(n, d, seed=17, amplitude=0.9)
    kap = np.exp(np.random.default_rng(2).normal(size=(n,) * d)) if kind == "ndk3d" else None
    lam = 4.0
    J = fem.assemble_jacobian(kind, u, lam, kap).toarray()
    m = fem.interior(u.shape).ravel()
    Jb = np.zeros_like(J)
    t = 1e-6
    for col in np.flatnonzero(m):
        e = np.zeros(u.size); e[col] = t
        e = e.reshape(u.shape)
        Jb[:, col] = ((fem.residual(kind, u + e, lam, kap) - fem.residual(kind, u - e, lam, kap)) / (2 * t)).ravel()
    assert np.max(np.abs(J - Jb)) <= 1e-8 * np.max(np.abs(J))


def test_bratu_jacobian_symmetric_nd_not():
    """Sec. 1: F = grad Psi makes J symmetric (Bratu); nonlinear diffusion is not
    a gradient, so J(u) is nonsymmetric away from u = 0."""
    ub = random_state_field(6, 2, seed=1)
    Jb = fem.assemble_jacobian("bratu2d", ub, 5.0)
    assert abs(Jb - Jb.T).max() <= 1e-15 * abs(Jb).max()
    un = random_state_field(4, 3, seed=1)
    Jn = fem.assemble_jacobian("nd3d", un)
    assert abs(Jn - Jn.T).max() >= 1e-3 * abs(Jn).max()
    J0 = fem.assemble_jacobian("nd3d", np.zeros_like(un))
    assert abs(J0 - J0.T).max() <= 1e-15 * abs(J0).max()


def test_residual_at_samples_matches_full():
    n = 7
    u = random_state_field(n, 3, seed=8, kind="mms", amplitude=0.1)
    b = fem.mms_load(n)
    F = fem.residual("nd3d", u, load=b)
    rng = np.random.default_rng(0)
    nodes = [tuple(rng.integers(0, n + 1, size=3)) for _ in range(20)]
    Fs = fem.residual_at("nd3d", u, nodes, load=b)
    assert np.allclose(Fs, [F[nd] for nd in nodes], rtol=1e-13, atol=1e-17)
    ub = random_state_field(n, 2, seed=8)
    Fb = fem.residual("bratu2d", ub, 3.0)
    nodes2 = [tuple(rng.integers(0, n + 1, size=2)) for _ in range(20)]
    assert np.allclose(fem.residual_at("bratu2d", ub, nodes2, lam=3.0), [Fb[nd] for nd in nodes2], rtol=1e-13, atol=1e-17)


def test_nd_manufactured_solution_converges_second_order():
    """The discrete solution approaches u* = sin(pi x) sin(pi y) sin(pi z) at O(h^2),
    which pins the nonlinear flux and the load vector together."""
    errs = []
    for n in (8, 16):
        b = fem.mms_load(n)
        u, hist = adjoint.newton_direct("nd3d", np.zeros((n + 1,) * 3), load=b, rtol=1e-12)
        x, y, z = fem.node_coords(n, 3)
        errs.append(np.max(np.abs(u - fem.mms_exact(x, y, z))))
    rate = np.log2(errs[0] / errs[1])
    assert 1.8 <= rate <= 2.3, (errs, rate)


def test_vjp_matches_assembled_transpose_and_kappa_derivative():
    n = 4
    u = random_state_field(n, 3, seed=21, amplitude=0.6)
    kap = np.exp(np.random.default_rng(4).normal(size=(n, n, n)))
    w = random_direction(n, 3, seed=22)
    JTw, dk = fem.vjp_ndk3d(u, kap, w)
    J = fem.assemble_jacobian("ndk3d", u, 0.0, kap)
    assert np.allclose(JTw.ravel(), J.T @ w.ravel(), rtol=1e-12, atol=1e-15)
    # F is linear in kappa_e: central difference along e_e is exact up to round-off
    m = fem.interior(u.shape)
    for e in [(0, 0, 0), (1, 2, 3), (3, 3, 3)]:
        kp = kap.copy(); kp[e] += 0.5
        km = kap.copy(); km[e] -= 0.5
        dF = fem.residual("ndk3d", u, kappa=kp) - fem.residual("ndk3d", u, kappa=km)
        assert abs(np.sum(dF[m] * w[m]) - dk[e]) <= 1e-12 * (abs(dk[e]) + 1e-12)


def test_mms_load_at_samples_matches_full():
    n = 6
    b = fem.mms_load(n)
    rng = np.random.default_rng(3)
    nodes = [tuple(rng.integers(0, n + 1, size=3)) for _ in range(25)]
    assert np.allclose(fem.mms_load_at(n, nodes), [b[nd] for nd in nodes], rtol=1e-13, atol=1e-18)
