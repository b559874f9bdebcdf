"""Pins of the oracle's backtracking line search (Dennis & Schnabel, Sec. 6.3;
used by the inexact Newton method of Sec. 3) on merit functions whose
minimisers are known in closed form.

The merit is phi(alpha) = 1/2 ||F(u + alpha du)||^2.  Each case uses a scalar
state u = 0, du = 1 and F(x) = sqrt(2 phi(x)), so phi is exactly the chosen
function of alpha, and passes phi'(0) as the slope."""
import numpy as np
import pytest

from oracle import jfnk

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _run(phi, slope, max_steps=10):
    F_of = lambda x: np.array([np.sqrt(2.0 * phi(float(x[0])))])  # noqa: E731
    trials = []
    alpha, Fn, ok = jfnk.backtrack(F_of, np.zeros(1), np.ones(1), F_of(np.zeros(1)), slope,
                                   max_steps=max_steps, trials=trials)
    return alpha, Fn, ok, trials


def test_full_step_accepted_when_it_decreases_enough():
    alpha, Fn, ok, trials = _run(lambda a: 1.0 - 0.5 * a, -0.5)
    assert ok and alpha == 1.0 and trials == [1.0]
    assert 0.5 * Fn[0] ** 2 == pytest.approx(0.5, rel=1e-14)


def test_quadratic_step_is_the_exact_minimiser_of_a_quadratic_merit():
    # phi = 1 - a + k a^2: the quadratic through phi(0), phi'(0), phi(1) is phi
    # itself, so the first backtrack lands on its minimiser 1/(2k)
    for k in (1.25, 2.5, 4.0):
        alpha, _, ok, trials = _run(lambda a: 1.0 - a + k * a * a, -1.0)
        assert ok and len(trials) == 2
        assert alpha == pytest.approx(1.0 / (2.0 * k), rel=1e-13)


def test_cubic_step_is_the_exact_minimiser_of_a_cubic_merit():
    # phi = 1 - a + 1000 a^3: the quadratic step 1/2000 is raised to the lower
    # bound 0.1 * 1; phi(0.1) = 1.9 fails; the cubic through phi(0), phi'(0),
    # phi(1), phi(0.1) is phi itself, whose local minimiser 1/sqrt(3000) lies
    # inside [0.01, 0.05] and is accepted
    alpha, Fn, ok, trials = _run(lambda a: 1.0 - a + 1000.0 * a ** 3, -1.0)
    assert ok and len(trials) == 3
    assert trials[1] == pytest.approx(0.1, rel=1e-15)
    assert alpha == pytest.approx(1.0 / np.sqrt(3000.0), rel=1e-12)
    assert 0.5 * Fn[0] ** 2 == pytest.approx(1.0 - 2.0 / (3.0 * np.sqrt(3000.0)), rel=1e-12)


def test_cubic_step_on_a_general_merit_matches_the_interpolating_cubic():
    # a non-polynomial merit: the second backtrack must be the stationary point
    # (local minimum) of the cubic interpolating phi(0), phi'(0) and the two
    # rejected trials, computed here from the 4x4 interpolation system
    phi = lambda a: np.exp(6.0 * a) - 7.0 * a  # noqa: E731
    slope = -1.0
    alpha, _, ok, trials = _run(phi, slope)
    assert len(trials) >= 3
    a1, a2 = trials[0], trials[1]
    M = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 1.0, 0.0, 0.0],
                  [1.0, a1, a1 ** 2, a1 ** 3], [1.0, a2, a2 ** 2, a2 ** 3]])
    coef = np.linalg.solve(M, np.array([phi(0.0), slope, phi(a1), phi(a2)]))
    roots = np.roots([3.0 * coef[3], 2.0 * coef[2], coef[1]])
    minima = [r.real for r in roots if abs(r.imag) == 0.0 and 6.0 * coef[3] * r.real + 2.0 * coef[2] > 0.0]
    assert len(minima) == 1
    t = min(max(minima[0], 0.1 * a2), 0.5 * a2)
    assert trials[2] == pytest.approx(t, rel=1e-10)


def test_new_step_is_clipped_to_at_most_half_the_previous():
    # phi(1) just above the Armijo line: the quadratic minimiser 1/(2k) is a
    # little above 0.5 and is cut to 0.5
    k = 1.0 - 0.5e-4
    alpha, _, ok, trials = _run(lambda a: 1.0 - a + k * a * a, -1.0)
    assert trials[:2] == [1.0, 0.5] and ok


def test_non_finite_trial_is_cut_to_a_tenth_and_not_interpolated():
    # phi is NaN beyond 0.05: alpha = 1 and 0.1 are cut by 10 each; 0.01 gives
    # a sufficient decrease
    phi = lambda a: float("nan") if a > 0.05 else 1.0 - a + a * a  # noqa: E731
    alpha, Fn, ok, trials = _run(phi, -1.0)
    assert ok and trials == pytest.approx([1.0, 0.1, 0.01], rel=1e-15)
    assert np.isfinite(Fn).all()


def test_exhaustion_returns_the_last_tested_step_with_its_own_residual():
    # a slope that is not a descent direction of phi (phi increases): no trial
    # can satisfy the Armijo condition; after max_steps trials the last tested
    # step comes back with its own residual
    phi = lambda a: 1.0 + a  # noqa: E731
    for m in (1, 3, 10):
        alpha, Fn, ok, trials = _run(phi, -1.0, max_steps=m)
        assert not ok and len(trials) == m
        assert alpha == trials[-1]
        assert 0.5 * Fn[0] ** 2 == pytest.approx(phi(alpha), rel=1e-14)
    # the successive steps stay inside [0.1, 0.5] of their predecessor
    for a, b in zip(trials, trials[1:]):
        assert 0.1 * a * (1 - 1e-15) <= b <= 0.5 * a * (1 + 1e-15)


def test_newton_stops_at_the_last_accepted_iterate_when_the_line_search_fails():
    # one backtracking step allowed on a strongly nonlinear diffusion problem
    # (load scaled so that the full Newton step from u = 0 overshoots): the solve
    # ends with status 'linesearch' and keeps u = u0
    from oracle import fem
    n = 8
    load = 40.0 * fem.mms_load(n)
    lv = jfnk.build_hierarchy("nd3d", n, 2, load=load)
    opts = jfnk.Options(nu_pre=2, nu_post=2, cheb_degree=4, ls_max=1, max_newton=5)
    u, st = jfnk.newton_solve(lv, np.zeros((n + 1,) * 3), opts)
    assert st.status == "linesearch" and not st.converged
    assert st.newton_its == 1 and st.alpha_hist == [0.0]
    assert np.array_equal(u, np.zeros_like(u))
    assert st.res_hist[0] == st.res_hist[1]


@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("its", [1, 4, 9])
def test_arnoldi_slope_equals_the_direct_product(precond, its):
    # the line-search slope F . (J dx) after one FGMRES cycle comes from the
    # Arnoldi relation A Z y = V Hbar y: with b = -F = beta v_0 it is
    # b . (A x) = beta (Hbar y)_0.  Against the product formed directly with a
    # dense nonsymmetric A (and a flexible right preconditioner M):
    rng = np.random.default_rng(11 + its)
    n = 40
    A = np.eye(n) * 4.0 + rng.normal(size=(n, n)) * 0.3
    M = np.eye(n) + rng.normal(size=(n, n)) * 0.05
    b = rng.normal(size=n)
    mask = np.ones(n, dtype=bool)
    info = {}
    x, k, _ = jfnk.gmres(lambda v: A @ v, b, mask, 1e-30, its, precond=(lambda v: M @ v) if precond else None,
                         info=info)
    assert k == its and info["cycles"] == 1
    direct = float(b @ (A @ x))
    assert info["beta"] * info["Hy0"] == pytest.approx(direct, rel=1e-12)
    # with a restart the relation covers only the last cycle
    info2 = {}
    jfnk.gmres(lambda v: A @ v, b, mask, 1e-30, 6, restart=3, info=info2)
    assert info2["cycles"] == 2
