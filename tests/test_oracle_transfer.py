"""Pins of the oracle's transfer operators (Sec. 2, "Transfer Operators"):
R = I^T as an adjoint identity, P = 2^-d I^T preserving constants, and the
Galerkin identities of nested Q1 spaces (I^T K_f I = K_c, I^T M_f I = M_c),
which fix the interpolation weights independently of how I is written."""
import numpy as np
import pytest

from oracle import fem, transfer
from workloads import random_direction, random_state_field


@pytest.mark.parametrize("d,n", [(2, 4), (2, 7), (3, 3), (3, 4)])
def test_restriction_is_transpose_of_prolongation(d, n):
    x = random_direction(2 * n, d, seed=1)
    y = random_direction(n, d, seed=2)
    lhs = np.sum(transfer.restrict(x) * y)
    rhs = np.sum(x * transfer.prolong(y))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 3)])
def test_projection_is_scaled_restriction_on_interior_vectors(d, n):
    x = random_direction(2 * n, d, seed=3)
    assert np.allclose(transfer.project(x), 2.0 ** (-d) * transfer.restrict(x), rtol=1e-15, atol=0)


@pytest.mark.parametrize("d,n", [(2, 6), (3, 4)])
def test_projection_preserves_constants(d, n):
    """Sec. 2: the factor 2^-d makes P preserve constant functions."""
    c = np.full((2 * n + 1,) * d, 3.25)
    p = transfer.project(c)
    assert np.allclose(p, 3.25, rtol=1e-15)


def test_prolongation_reproduces_coarse_values_and_is_local():
    n = 4
    c = np.zeros((n + 1, n + 1))
    c[2, 1] = 1.0
    f = transfer.prolong(c)
    # a single coarse hat prolongates to the coarse hat sampled on the fine grid
    t = np.linspace(0, 1, 2 * n + 1)
    Y, X = np.meshgrid(t, t, indexing="ij")
    hat = np.clip(1 - np.abs(X - 1 / n) * n, 0, None) * np.clip(1 - np.abs(Y - 2 / n) * n, 0, None)
    assert np.allclose(f, hat, atol=1e-15)


@pytest.mark.parametrize("kind,n", [("bratu2d", 4), ("nd3d", 3)])
def test_galerkin_identity_nested_q1(kind, n):
    """For nested Q1 spaces the coarse linearised operator at u = 0 equals
    I^T J_fine(0) I exactly (stiffness and mass are integrated exactly)."""
    d = fem.dim_of(kind)
    lam = 2.0
    Jf = fem.assemble_jacobian(kind, np.zeros((2 * n + 1,) * d), lam).toarray()
    Jc = fem.assemble_jacobian(kind, np.zeros((n + 1,) * d), lam).toarray()
    m = fem.interior((n + 1,) * d).ravel()
    P = np.zeros((Jf.shape[0], Jc.shape[0]))
    for k in np.flatnonzero(m):
        e = np.zeros(Jc.shape[0]); e[k] = 1.0
        P[:, k] = transfer.prolong(e.reshape((n + 1,) * d)).ravel()
    G = P.T @ Jf @ P
    assert np.max(np.abs(G - Jc)) <= 1e-13 * np.max(np.abs(Jc))


def test_coarsen_kappa_mean():
    k = np.arange(64, dtype=float).reshape(4, 4, 4)
    c = transfer.coarsen_kappa(k)
    assert c.shape == (2, 2, 2)
    assert c[0, 0, 0] == np.mean(k[:2, :2, :2])
    assert c[1, 0, 1] == np.mean(k[2:, :2, 2:])


def test_random_state_boundary_zero():
    u = random_state_field(5, 3, seed=0, kind="mms", amplitude=0.1)
    assert np.all(u[fem.boundary_mask(u.shape)] == 0)
