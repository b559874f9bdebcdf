"""Property checks of the oracle over randomly drawn grid sizes and states
(hypothesis): identities the definitions fix for every size, so a mistake that
the fixed-size pins happen to miss (an index or sign that only matters on some
grids) fails here.  CPU only."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import fem, hyper, transfer  # noqa: E402

SETTINGS = settings(max_examples=15, deadline=None, derandomize=True)


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@SETTINGS
@given(d=st.sampled_from([2, 3]), nc=st.integers(1, 6), seed=st.integers(0, 10 ** 6))
def test_restriction_is_the_transpose_of_prolongation(d, nc, seed):
    """Sec. 2: R = I^T, i.e. <R r, c> = <r, I c> on every pair of grids (boundary
    entries are zero on both sides)."""
    r = _rand((2 * nc + 1,) * d, seed)
    c = _rand((nc + 1,) * d, seed + 1)
    r[fem.boundary_mask(r.shape)] = 0.0
    c[fem.boundary_mask(c.shape)] = 0.0
    lhs = float(np.sum(transfer.restrict(r) * c))
    rhs = float(np.sum(r * transfer.prolong(c)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(r).sum() * np.abs(c).max())


@SETTINGS
@given(d=st.sampled_from([2, 3]), nc=st.integers(1, 6), a=st.floats(-2.0, 2.0))
def test_projection_keeps_constants_at_interior_coarse_nodes(d, nc, a):
    """Sec. 2: P = 2^-d I^T preserves constants (at every interior coarse node)."""
    x = np.full((2 * nc + 1,) * d, a)
    p = transfer.project(x)
    assert np.allclose(p[fem.interior(p.shape)], a, rtol=0, atol=1e-14 * max(1.0, abs(a)))


@SETTINGS
@given(n=st.integers(2, 12), seed=st.integers(0, 10 ** 6), alpha=st.floats(-3.0, 3.0),
       beta=st.floats(-3.0, 3.0))
def test_bratu_residual_without_source_is_linear(n, seed, alpha, beta):
    """Sec. 3 (Bratu) with lambda = 0 is the Q1 Laplacian: F is linear in u."""
    u, w = _rand((n + 1, n + 1), seed), _rand((n + 1, n + 1), seed + 1)
    lhs = fem.residual("bratu2d", alpha * u + beta * w, 0.0)
    rhs = alpha * fem.residual("bratu2d", u, 0.0) + beta * fem.residual("bratu2d", w, 0.0)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * (1.0 + np.abs(rhs).max()))


@SETTINGS
@given(n=st.integers(2, 8), seed=st.integers(0, 10 ** 6))
def test_nonlinear_diffusion_commutes_with_axis_permutations(n, seed):
    """The ND operator -div((1+u^2) grad u) on the cube and its Q1/Gauss
    discretisation are invariant under permutations of the axes."""
    u = _rand((n + 1,) * 3, seed) * 0.5
    A = fem.operator("nd3d", u)
    for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1)):
        Ap = fem.operator("nd3d", np.transpose(u, perm))
        assert np.allclose(Ap, np.transpose(A, perm), rtol=0, atol=1e-13 * (1.0 + np.abs(A).max()))


@SETTINGS
@given(n=st.integers(2, 10), seed=st.integers(0, 10 ** 6))
def test_minimal_surface_is_invariant_under_adding_a_constant(n, seed):
    """Sec. 3 (minimal surface): the area depends on grad u only, so u + c has
    the same residual."""
    u = _rand((n + 1, n + 1), seed) * 0.3
    F0 = fem.residual("minsurf2d", u)
    F1 = fem.residual("minsurf2d", u + 0.7)
    assert np.allclose(F0, F1, rtol=0, atol=1e-12 * (1.0 + np.abs(F0).max()))


@SETTINGS
@given(m=st.integers(1, 2), seed=st.integers(0, 10 ** 6), shift=st.floats(-0.5, 0.5))
def test_beam_residual_is_invariant_under_rigid_translation(m, seed, shift):
    """Sec. 3 (hyperelasticity): W depends on F = I + grad u only, so a uniform
    translation of every node (Dirichlet data included) leaves the residual
    unchanged."""
    u = hyper.boundary_state(m)
    mask = hyper.unknown_mask(u.shape)
    u[mask] += 0.1 / m * np.random.default_rng(seed).uniform(-1.0, 1.0, size=int(mask.sum()))
    t = np.array([shift, -0.5 * shift, 0.25 * shift])
    F0, F1 = hyper.residual(u), hyper.residual(u + t)
    assert np.allclose(F0, F1, rtol=0, atol=1e-11 * (1.0 + np.abs(F0).max()))
