"""Transfer operators between nested structured Q1 grids (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Sec. 2 ("Transfer Operators") defines the interpolation I (coarse -> fine),
the restriction R = I^T and the projection of the Newton iterate
P = 2^-d I^T; the factor 2^-d makes P preserve constant functions.

Coarse grid n elements per direction, fine grid 2n.  Coarse node i coincides
with fine node 2i.  I is the Q1 interpolation: in 1D fine[2i] = c[i] and
fine[2i+1] = (c[i] + c[i+1]) / 2, and the d-dimensional I is the tensor
product of the 1D one.

Readings where the paper is silent (all vectors are full node grids):
  * prolong: the coarse boundary entries are corrections of Dirichlet values and
    are taken as 0; fine boundary entries of the result are 0.
  * restrict: fine boundary entries of a residual are 0 by convention (they are
    zeroed before the transpose is applied); coarse boundary entries are 0.
  * project: interior coarse nodes take 2^-d (I^T x) over the whole fine grid,
    boundary values included, so P maps the constant 1 to 1 at every interior
    coarse node; coarse boundary nodes take the coincident fine value
    (injection of the Dirichlet data).  For the homogeneous Dirichlet data of
    every configuration here this equals applying 2^-d I^T to interior values.
"""
import numpy as np

from .fem import boundary_mask


def interp_matrix_1d(n):
    """(2n+1) x (n+1) dense 1D interpolation matrix of nested linear elements."""
    M = np.zeros((2 * n + 1, n + 1))
    for i in range(n + 1):
        M[2 * i, i] = 1.0
    for i in range(n):
        M[2 * i + 1, i] = 0.5
        M[2 * i + 1, i + 1] = 0.5
    return M


def _apply_each_axis(x, mats):
    """Apply matrix mats[ax] along every array axis ax of x."""
    y = x
    for ax, M in enumerate(mats):
        y = np.moveaxis(np.tensordot(M, np.moveaxis(y, ax, 0), axes=(1, 0)), 0, ax)
    return y


def prolong(c):
    """I c: coarse correction (n+1)^d -> fine (2n+1)^d, boundary zero."""
    c = np.where(boundary_mask(c.shape), 0.0, c)
    n = c.shape[0] - 1
    M = interp_matrix_1d(n)
    f = _apply_each_axis(c, [M] * c.ndim)
    f[boundary_mask(f.shape)] = 0.0
    return f


def restrict(r):
    """R r = I^T r: fine residual (2n+1)^d -> coarse (n+1)^d, boundary zero."""
    r = np.where(boundary_mask(r.shape), 0.0, r)
    n = (r.shape[0] - 1) // 2
    M = interp_matrix_1d(n)
    c = _apply_each_axis(r, [M.T] * r.ndim)
    c[boundary_mask(c.shape)] = 0.0
    return c


def project(x):
    """P x = 2^-d I^T x on interior coarse nodes; injection on the coarse boundary."""
    d = x.ndim
    n = (x.shape[0] - 1) // 2
    M = interp_matrix_1d(n)
    c = _apply_each_axis(x, [M.T] * d) * 2.0 ** (-d)
    bm = boundary_mask(c.shape)
    inj = x[tuple(slice(None, None, 2) for _ in range(d))]
    c[bm] = inj[bm]
    return c


def coarsen_kappa(kappa):
    """Per-element coefficient on the coarse grid: arithmetic mean of the 2^d
    fine children (reading: the paper rediscretises each level and has no
    coefficient field; the mean is the simplest consistent choice)."""
    d = kappa.ndim
    n = kappa.shape[0] // 2
    acc = np.zeros((n,) * d)
    import itertools
    for o in itertools.product((0, 1), repeat=d):
        acc += kappa[tuple(slice(oo, None, 2) for oo in o)]
    return acc / 2 ** d
