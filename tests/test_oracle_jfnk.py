"""Pins of the oracle's Jacobian-free method against facts fixed outside it:
the analytic Jacobian (FD action), closed-form spectra (power method,
Chebyshev error polynomial), direct solves (coarse GMRES, Newton), counting
identities of Alg. 1 and the invariants the paper states (Sec. 3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

from oracle import adjoint, fem, jfnk, splitmix
from workloads import random_direction, random_state_field


def _eig_1d(n):
    th = np.arange(1, n) * np.pi / n
    return np.sin(th / 2) ** 2, 2.0 + np.cos(th)


def _sine_mode(n, d, modes):
    t = np.linspace(0.0, 1.0, n + 1)
    grids = np.meshgrid(*([t] * d), indexing="ij")
    v = np.ones((n + 1,) * d)
    for g, m in zip(reversed(grids), modes):
        v = v * np.sin(m * np.pi * g)
    v[fem.boundary_mask(v.shape)] = 0.0
    return v


def _nd_lambda_max(n):
    s, c = _eig_1d(n)
    h = 1.0 / n
    S, Cc = s[:, None, None], c[:, None, None]
    mu = 4 * h / 9 * (S * c[None, :, None] * c[None, None, :] + Cc * s[None, :, None] * c[None, None, :]
                      + Cc * c[None, :, None] * s[None, None, :])
    return mu.max()


def test_eps_closed_form_special_case():
    """x = 0, v = 1 on the n interior nodes: eps = sqrt(eps_p) / sqrt(n) (Sec. 1)."""
    n = 6
    mask = fem.interior((n + 1, n + 1))
    v = np.where(mask, 1.0, 0.0)
    e = jfnk.fd_eps(np.zeros_like(v), v, mask, "paper")
    assert e == pytest.approx(np.sqrt(2.0 ** -52) / np.sqrt(mask.sum()), rel=1e-15)
    e32 = jfnk.fd_eps(np.zeros_like(v), v, mask, "fp32")
    assert e32 == pytest.approx(np.sqrt(2.0 ** -23) / np.sqrt(mask.sum()), rel=1e-15)
    assert jfnk.fd_eps(np.zeros_like(v), np.zeros_like(v), mask) == 0.0


@pytest.mark.parametrize("kind,n", [("bratu2d", 24), ("nd3d", 8), ("ndk3d", 6)])
def test_fd_jv_matches_analytic_jacobian(kind, n):
    """The FD action approximates the assembled analytic J v to truncation O(eps)
    plus round-off O(eps_p / eps): both far below 1e-6 relative."""
    d = fem.dim_of(kind)
    u = random_state_field(n, d, seed=31, amplitude=0.8)
    kap = np.exp(np.random.default_rng(5).normal(size=(n,) * d)) if kind == "ndk3d" else None
    load = fem.mms_load(n) if kind == "nd3d" else None
    lv = jfnk.Level(kind, n, 5.0, kap, load)
    v = random_direction(n, d, seed=32)
    Fu = lv.F(u)
    Jv = jfnk.fd_jv(lv, u, Fu, v)
    Jex = (fem.assemble_jacobian(kind, u, 5.0, kap) @ v.ravel()).reshape(u.shape)
    assert np.linalg.norm(Jv - Jex) <= 1e-6 * np.linalg.norm(Jex)
    # the fp32-style step is much larger: truncation dominates but stays small
    Jv32 = jfnk.fd_jv(lv, u, Fu, v, mode="fp32")
    assert np.linalg.norm(Jv32 - Jex) <= 2e-3 * np.linalg.norm(Jex)


def test_power_method_bounded_by_and_converges_to_closed_form():
    """J(0) = K for nonlinear diffusion: ||K v|| <= lambda_max for unit v, and the
    power iteration approaches the closed-form lambda_max."""
    n = 8
    lv = jfnk.Level("nd3d", n, 0.0, None, None)
    x = np.zeros((n + 1,) * 3)
    Fx = lv.F(x)
    lmax = _nd_lambda_max(n)
    v0 = splitmix.start_vector(x.shape, 0, 1)
    lam10, _ = jfnk.power_method(lv, x, Fx, v0, 10)
    assert 0.7 * lmax <= lam10 <= lmax * (1 + 1e-7)
    lam300, _ = jfnk.power_method(lv, x, Fx, v0, 300)
    assert abs(lam300 - lmax) <= 2e-3 * lmax
    # the paper's stopping rule terminates early with a close estimate
    lam_tol, _ = jfnk.power_method(lv, x, Fx, v0, 30, tol=1e-2)
    assert 0.7 * lmax <= lam_tol <= lmax * (1 + 1e-7)


@pytest.mark.parametrize("degree,nu", [(3, 1), (4, 2), (3, 3)])
def test_chebyshev_error_polynomial_on_eigenmodes(degree, nu):
    """Linear limit: for J s = mu v with sine eigenvector v the smoothed iterate
    from s = 0 is (1 - p(mu)^nu) v with p(t) = T_k((theta - t)/delta) / T_k(theta/delta)
    (Chebyshev polynomial from numpy, independent of the recurrence)."""
    n = 8
    lv = jfnk.Level("nd3d", n, 0.0, None, None)
    x = np.zeros((n + 1,) * 3)
    Fx = lv.F(x)
    lmax = _nd_lambda_max(n)
    s1, c1 = _eig_1d(n)
    h = 1.0 / n
    a_, b_ = 0.1 * lmax, 1.1 * lmax
    theta, delta = (a_ + b_) / 2, (b_ - a_) / 2
    Tk = np.zeros(degree + 1); Tk[-1] = 1.0
    for modes in [(1, 1, 1), (4, 3, 5), (7, 7, 7)]:
        v = _sine_mode(n, 3, modes)
        i, j, k = [m - 1 for m in modes]
        mu = 4 * h / 9 * (s1[i] * c1[j] * c1[k] + c1[i] * s1[j] * c1[k] + c1[i] * c1[j] * s1[k])
        s = jfnk.chebyshev(lv, np.zeros_like(x), x, Fx, mu * v, nu, degree, lmax, 0.1, 1.1)
        p = C.chebval((theta - mu) / delta, Tk) / C.chebval(theta / delta, Tk)
        expect = (1 - p ** nu) * v
        assert np.max(np.abs(s - expect)) <= 1e-6 * np.max(np.abs(v))


def test_coarse_gmres_n0_iterations_equals_direct_solve():
    """Unrestarted GMRES run for n_0 iterations on an n_0-dimensional system is
    the exact solve; with the FD action it matches the analytic direct solve up
    to the FD error."""
    n = 4
    u = random_state_field(n, 3, seed=41, amplitude=0.5)
    lv = jfnk.Level("nd3d", n, 0.0, None, None)
    Fu = lv.F(u)
    b = random_direction(n, 3, seed=42)
    s, its, _ = jfnk.gmres(lambda v: jfnk.fd_jv(lv, u, Fu, v), b, lv.mask, 1e-14, lv.n_unknowns)
    J = fem.assemble_jacobian("nd3d", u)
    m = lv.mask.ravel()
    idx = np.flatnonzero(m)
    x = np.zeros(u.size)
    x[idx] = spla.spsolve(J[idx][:, idx].tocsc(), b.ravel()[idx])
    assert np.linalg.norm(s.ravel() - x) <= 1e-6 * np.linalg.norm(x)
    # exact linear operator: GMRES reproduces the direct solve to round-off
    A = lambda v: (J @ v.ravel()).reshape(v.shape)
    s2, _, _ = jfnk.gmres(A, b, lv.mask, 1e-15, lv.n_unknowns)
    assert np.linalg.norm(s2.ravel() - x) <= 1e-10 * np.linalg.norm(x)


def test_fgmres_with_exact_preconditioner_converges_in_one_iteration():
    n = 6
    u = random_state_field(n, 2, seed=5)
    J = fem.assemble_jacobian("bratu2d", u, 3.0)
    m = fem.interior(u.shape).ravel()
    idx = np.flatnonzero(m)
    Ji = J[idx][:, idx].tocsc()
    A = lambda v: (J @ v.ravel()).reshape(v.shape)

    def Minv(v):
        x = np.zeros(v.size)
        x[idx] = spla.spsolve(Ji, v.ravel()[idx])
        return x.reshape(v.shape)
    b = random_direction(n, 2, seed=6)
    x, its, res = jfnk.gmres(A, b, fem.interior(u.shape), 1e-10, 50, precond=Minv, restart=30)
    assert its == 1 and res <= 1e-10 * np.linalg.norm(b)
    # with the identity preconditioner FGMRES is GMRES
    x1, it1, _ = jfnk.gmres(A, b, fem.interior(u.shape), 1e-8, 200, precond=lambda v: v, restart=30)
    x2, it2, _ = jfnk.gmres(A, b, fem.interior(u.shape), 1e-8, 200, restart=30)
    assert it1 == it2 and np.allclose(x1, x2, rtol=1e-12, atol=1e-14)


def test_vcycle_counts_gradient_evaluations_per_alg1():
    """Alg. 1 with V(3,3), degree 3: on each smoothed level a cycle costs
    pre 2+3+3, restriction 1, post 3+3+3 = 18 FD actions (one F each)."""
    n, L = 32, 3
    lv = jfnk.build_hierarchy("bratu2d", n, L, lam=5.0)
    o = jfnk.Options(nu_pre=3, nu_post=3, cheb_degree=3)
    u = np.zeros((n + 1, n + 1))
    jfnk.setup_levels(lv, u, o, 0)
    before = [x.ge for x in lv]
    b = random_direction(n, 2, seed=1)
    jfnk.mg_vcycle(lv, L - 1, b, o)
    used = [x.ge - y for x, y in zip(lv, before)]
    assert used[1] == 18 and used[2] == 18
    assert 1 <= used[0] <= lv[0].n_unknowns


@pytest.mark.parametrize("n", [16, 32, 64])
def test_vcycle_contraction_level_independent(n):
    """Sec. 3: the multigrid preconditioner is level-independent.  As a
    stationary iteration on the linearised Bratu problem its error contraction
    stays well below 1 and does not grow with n."""
    levels = int(np.log2(n)) - 1
    lv = jfnk.build_hierarchy("bratu2d", n, levels, lam=5.0)
    o = jfnk.Options()
    u = np.zeros((n + 1, n + 1))
    jfnk.setup_levels(lv, u, o, 0)
    fine = lv[-1]
    J = fem.assemble_jacobian("bratu2d", u, 5.0)
    xs = random_direction(n, 2, seed=9)
    b = (J @ xs.ravel()).reshape(u.shape)
    x = np.zeros_like(u)
    errs = []
    for _ in range(4):
        r = b - (J @ x.ravel()).reshape(u.shape)
        x = x + jfnk.mg_vcycle(lv, levels - 1, r, o)
        errs.append(np.linalg.norm(x - xs))
    rho = (errs[-1] / errs[0]) ** (1 / 3)
    assert rho < 0.15, rho


def test_newton_quadratic_and_matches_direct_solution():
    """Bratu lambda = 5, 64^2 elements, 4 levels: the JFNK-MG solution equals the
    exact-Newton discrete solution, the final steps contract quadratically and
    the solution has the square's symmetry."""
    n = 64
    lv = jfnk.build_hierarchy("bratu2d", n, 4, lam=5.0)
    o = jfnk.Options(rtol_newton=1e-11)
    u, st = jfnk.newton_solve(lv, np.zeros((n + 1, n + 1)), o)
    assert st.converged and st.newton_its <= 6
    ud, _ = adjoint.newton_direct("bratu2d", np.zeros((n + 1, n + 1)), lam=5.0)
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
    assert np.max(np.abs(ud - ud.T)) <= 1e-12 and np.max(np.abs(ud - ud[:, ::-1])) <= 1e-12
    # ||F_{k+1}|| <= C ||F_k||^2 over the steps above the FD round-off floor
    # (the sqrt(eps_p)-accurate FD action limits the last step near 1e-11 ||F_0||)
    r = [x for x in st.res_hist if x > 1e-9 * st.res_hist[0]]
    consts = [r[i + 1] / r[i] ** 2 for i in range(1, len(r) - 1)]
    assert len(consts) >= 2 and max(consts) <= 10.0, consts


def test_bratu_newton_count_constant_under_refinement():
    """Sec. 3: the number of inexact Newton iterations for Bratu does not depend
    on the refinement level."""
    counts = []
    for n, L in [(16, 2), (32, 3), (64, 4), (128, 5)]:
        lv = jfnk.build_hierarchy("bratu2d", n, L, lam=5.0)
        _, st = jfnk.newton_solve(lv, np.zeros((n + 1, n + 1)), jfnk.Options(rtol_newton=1e-8))
        counts.append(st.newton_its)
    assert max(counts) - min(counts) <= 1, counts


def test_ge_formula_weights():
    lv = jfnk.build_hierarchy("nd3d", 8, 3)
    for l, x in enumerate(lv):
        x.ge = 10 * (l + 1)
    # GE = sum 2^{-d(L-l)} GE_l with d = 3, L = 2: 10/64 + 20/8 + 30
    assert jfnk.total_ge(lv) == pytest.approx(10 / 64 + 20 / 8 + 30)


def test_splitmix_counter_form_equals_sequential_stream():
    seq = splitmix.sequential(12345, 50)
    with np.errstate(over="ignore"):
        z = np.uint64(12345) + (np.arange(50, dtype=np.uint64) + np.uint64(1)) * splitmix.GAMMA
    ctr = splitmix.finalise(z)
    assert [int(a) for a in ctr] == seq
    v = splitmix.uniform_pm1(7, 2, np.arange(200000, dtype=np.uint64))
    assert -1.0 <= v.min() and v.max() < 1.0
    assert abs(v.mean()) < 0.01 and abs(v.var() - 1.0 / 3.0) < 0.01


def test_power_method_stopping_rule_on_two_eigenmodes():
    """The Sec. 2 stopping rule (stop once successive estimates differ by less
    than tol, read relative to the newer one, after at least two iterations).
    Linear limit x = 0, J = K, start vector alpha e_A + beta e_B of two
    orthonormal sine eigenvectors: the k-th estimate is
    sqrt(a^2 mu_A^2k + b^2 mu_B^2k) / sqrt(a^2 mu_A^2(k-1) + b^2 mu_B^2(k-1)),
    so the iteration where the rule stops, and the estimate it returns, follow
    in closed form."""
    n = 8
    h = 1.0 / n
    lv = jfnk.Level("nd3d", n, 0.0, None, None)
    x = np.zeros((n + 1,) * 3)
    Fx = lv.F(x)
    s, c = _eig_1d(n)

    def mu(i, j, k):
        return 4 * h / 9 * (s[i - 1] * c[j - 1] * c[k - 1] + c[i - 1] * s[j - 1] * c[k - 1]
                            + c[i - 1] * c[j - 1] * s[k - 1])

    mA, mB = (3, 2, 1), (1, 2, 1)
    muA, muB = mu(*mA), mu(*mB)
    eA, eB = _sine_mode(n, 3, mA), _sine_mode(n, 3, mB)
    eA, eB = eA / np.linalg.norm(eA), eB / np.linalg.norm(eB)
    assert abs(np.vdot(eA, eB)) < 1e-14
    # the modes are eigenvectors of the linearised operator
    for e, m in ((eA, muA), (eB, muB)):
        Je = jfnk.fd_jv(lv, x, Fx, e)
        assert np.linalg.norm(Je - m * e) <= 1e-7 * m
    al, be = 0.3, 1.0
    lam = [np.sqrt(al ** 2 * muA ** (2 * k) + be ** 2 * muB ** (2 * k))
           / np.sqrt(al ** 2 * muA ** (2 * k - 2) + be ** 2 * muB ** (2 * k - 2)) for k in range(1, 40)]
    stops = []
    for tol in (1e-2, 1e-3, 1e-4):
        K = next(k for k in range(1, len(lam)) if abs(lam[k] - lam[k - 1]) < tol * lam[k])
        stops.append(K)
        # the closed-form sequence decides the stop with a clear margin
        assert abs(lam[K] - lam[K - 1]) < 0.95 * tol * lam[K]
        assert K < 2 or abs(lam[K - 1] - lam[K - 2]) > 1.05 * tol * lam[K - 1]
        got, _ = jfnk.power_method(lv, x, Fx, al * eA + be * eB, 30, tol=tol)
        assert got == pytest.approx(lam[K], rel=1e-7)
        assert abs(lam[K] - lam[K + 1]) > 100 * 1e-7 * lam[K] and abs(lam[K] - lam[K - 1]) > 100 * 1e-7 * lam[K]
    assert stops[0] < stops[1] < stops[2] < 29
    # the iteration cap wins over the rule
    got, _ = jfnk.power_method(lv, x, Fx, al * eA + be * eB, 2, tol=1e-12)
    assert got == pytest.approx(lam[1], rel=1e-7)
