"""Neo-Hookean hyperelastic beam of Sec. 3 ("Hyperelasticity") -- oracle.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Problem (Sec. 3): Omega = (0,10) x (0,1) x (0,1), displacement u in R^3,
  Psi_N(u) = int mu/2 (I_C - 3) - mu ln J + lam/2 (ln J)^2 dx,
  F = I + grad u, J = det F, I_C = tr(F^T F),
  mu = E / (2 (1+nu)), lam = E nu / ((1+nu)(1-2nu)), E = 10, nu = 0.3,
  u = 0 on x = 0 and u = u2(y, z) on x = 10 with
  u2 = (0, (0.5 + (y-1/2) cos(pi/6) - (z-1/2) sin(pi/6) - y) / 2,
          (0.5 + (y-1/2) sin(pi/6) + (z-1/2) cos(pi/6) - z) / 2),
  the other faces traction free.

Readings (the paper fixes the mesh family and "first order FE"):
  * Q1 hexahedra on the refinement-level grid of 10 m x m x m elements
    (m = 2^k; T_0 is 10 x 1 x 1), i.e. cubes of side h = 1/m, 2x2x2 Gauss rule.
  * Nodal arrays have shape (m+1, m+1, 10m+1, 3): axes z, y, x, component.
  * Unknowns: the 3 components at every node with 0 < x < 10 (the y and z
    faces are free); residual entries at the Dirichlet faces are 0.
  * F_a = int P(F) grad phi_a with the first Piola-Kirchhoff stress
    P = dW/dF = mu F + (lam ln J - mu) F^-T: the gradient of the discrete energy.
  * Projection of the iterate (Sec. 2, P = 2^-d I^T "so that constants are
    preserved"): on the free faces a coarse node has fewer fine neighbours, and
    2^-d I^T would not preserve constants there; each row of I^T is divided by
    its sum instead, which is 2^d at every node away from the free faces (the
    paper's operator there).  The Dirichlet faces take the injected data.
  * Initial guess: the Dirichlet data, 0 elsewhere.
"""
import itertools

import numpy as np

from .transfer import interp_matrix_1d

E_MOD = 10.0
NU = 0.3
MU = E_MOD / (2.0 * (1.0 + NU))
LAMBDA = E_MOD * NU / ((1.0 + NU) * (1.0 - 2.0 * NU))
LENGTH = 10
GAUSS_A = 1.0 / np.sqrt(3.0)
QP1 = np.array([0.5 - 0.5 * GAUSS_A, 0.5 + 0.5 * GAUSS_A])


def shape_of(m):
    """Node array shape of refinement level m = 2^k: (z, y, x, component)."""
    return (m + 1, m + 1, LENGTH * m + 1, 3)


def node_coords(m):
    """(x, y, z) coordinate arrays of shape (m+1, m+1, 10m+1)."""
    h = 1.0 / m
    z, y, x = np.meshgrid(np.arange(m + 1) * h, np.arange(m + 1) * h, np.arange(LENGTH * m + 1) * h,
                          indexing="ij")
    return x, y, z


def end_displacement(y, z):
    """u2(y, z) of Sec. 3 on the face x = 10."""
    c, s = np.cos(np.pi / 6.0), np.sin(np.pi / 6.0)
    return np.stack([np.zeros_like(y),
                     0.5 * (0.5 + (y - 0.5) * c - (z - 0.5) * s - y),
                     0.5 * (0.5 + (y - 0.5) * s + (z - 0.5) * c - z)], axis=-1)


def dirichlet_mask(shape):
    """True at the components of the nodes on x = 0 and x = 10."""
    m = np.zeros(shape, dtype=bool)
    m[:, :, 0, :] = True
    m[:, :, -1, :] = True
    return m


def unknown_mask(shape):
    """True at the unknown components: every node with 0 < x < 10 (the lateral
    faces are traction free, Sec. 3)."""
    return ~dirichlet_mask(shape)


def boundary_state(m):
    """Node array with the Dirichlet data (u = 0 at x = 0, u2 at x = 10), 0 elsewhere."""
    u = np.zeros(shape_of(m))
    x, y, z = node_coords(m)
    u[:, :, -1, :] = end_displacement(y[:, :, -1], z[:, :, -1])
    return u


def _m_of(shape):
    return shape[0] - 1


# ---------------------------------------------------------------------------
# Element routine
# ---------------------------------------------------------------------------

def _local_offsets():
    return list(itertools.product((0, 1), repeat=3))  # (ox, oy, oz)


def _gather(u):
    """Dict local offset (ox, oy, oz) -> array (m, m, 10m, 3) of nodal displacements."""
    mz, my, mx = u.shape[0] - 1, u.shape[1] - 1, u.shape[2] - 1
    return {o: u[o[2]:o[2] + mz, o[1]:o[1] + my, o[0]:o[0] + mx, :] for o in _local_offsets()}


def _scatter_add(out, contrib):
    mz, my, mx = out.shape[0] - 1, out.shape[1] - 1, out.shape[2] - 1
    for o, c in contrib.items():
        out[o[2]:o[2] + mz, o[1]:o[1] + my, o[0]:o[0] + mx, :] += c
    return out


def _grad_phi(o, xi, h):
    """Physical gradient (d/dx, d/dy, d/dz) of the trilinear shape function of local node o."""
    def s(oo, t):
        return 1.0 - t if oo == 0 else t

    def ds(oo):
        return -1.0 if oo == 0 else 1.0

    return np.array([ds(o[0]) * s(o[1], xi[1]) * s(o[2], xi[2]),
                     s(o[0], xi[0]) * ds(o[1]) * s(o[2], xi[2]),
                     s(o[0], xi[0]) * s(o[1], xi[1]) * ds(o[2])]) / h


def _gauss():
    for i, j, k in itertools.product(range(2), repeat=3):
        yield (QP1[i], QP1[j], QP1[k]), 0.125


def deformation_gradients(u):
    """Yield (weight * volume, F, {offset: grad phi}) at every Gauss point, F of
    shape (m, m, 10m, 3, 3) with F[..., i, j] = delta_ij + d u_i / d x_j."""
    m = _m_of(u.shape)
    h = 1.0 / m
    U = _gather(u)
    for xi, w in _gauss():
        G = {o: _grad_phi(o, xi, h) for o in U}
        F = np.zeros(next(iter(U.values())).shape[:3] + (3, 3))
        for o, g in G.items():
            F += U[o][..., :, None] * g[None, None, None, None, :]
        F += np.eye(3)
        yield w * h ** 3, F, G


def energy_density(F):
    """W(F) = mu/2 (I_C - 3) - mu ln J + lam/2 (ln J)^2 (Sec. 3); +inf where J <= 0."""
    J = np.linalg.det(F)
    IC = np.einsum("...ij,...ij->...", F, F)
    with np.errstate(invalid="ignore", divide="ignore"):
        lnJ = np.where(J > 0.0, np.log(np.where(J > 0.0, J, 1.0)), np.nan)
    W = 0.5 * MU * (IC - 3.0) - MU * lnJ + 0.5 * LAMBDA * lnJ ** 2
    return np.where(J > 0.0, W, np.inf)


def first_piola(F):
    """P = dW/dF = mu F + (lam ln J - mu) F^-T."""
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    with np.errstate(invalid="ignore"):
        lnJ = np.log(J)
    return MU * F + (LAMBDA * lnJ - MU)[..., None, None] * FinvT


def energy(u):
    """Discrete energy Psi_N(u_h) with the 2x2x2 Gauss rule."""
    total = 0.0
    for wv, F, _ in deformation_gradients(u):
        total += wv * float(np.sum(energy_density(F)))
    return total


def residual(u):
    """F_a = int P(F) grad phi_a (all 3 components), 0 at the Dirichlet nodes."""
    out = np.zeros(u.shape)
    for wv, F, G in deformation_gradients(u):
        P = first_piola(F)
        contrib = {o: wv * np.einsum("...ij,j->...i", P, g) for o, g in G.items()}
        _scatter_add(out, contrib)
    out[dirichlet_mask(u.shape)] = 0.0
    return out


def linear_elastic_residual(w):
    """Independent small-strain operator K_lin w = int sigma(eps(w)) grad phi_a,
    sigma = lam tr(eps) I + 2 mu eps (the linearisation of P at F = I)."""
    m = _m_of(w.shape)
    h = 1.0 / m
    W = _gather(w)
    out = np.zeros(w.shape)
    for xi, wq in _gauss():
        G = {o: _grad_phi(o, xi, h) for o in W}
        gw = sum(W[o][..., :, None] * G[o][None, None, None, None, :] for o in W)
        eps = 0.5 * (gw + np.swapaxes(gw, -1, -2))
        tr = np.trace(eps, axis1=-2, axis2=-1)
        sig = LAMBDA * tr[..., None, None] * np.eye(3) + 2.0 * MU * eps
        _scatter_add(out, {o: wq * h ** 3 * np.einsum("...ij,j->...i", sig, g) for o, g in G.items()})
    out[dirichlet_mask(w.shape)] = 0.0
    return out


# ---------------------------------------------------------------------------
# Transfers between the level grids (coarse m, fine 2m)
# ---------------------------------------------------------------------------

def _axis_mats(mc):
    """1D interpolation matrices for the z, y, x axes of a coarse grid with m = mc."""
    return [interp_matrix_1d(mc), interp_matrix_1d(mc), interp_matrix_1d(LENGTH * mc)]


def _apply_axes(x, mats):
    y = x
    for ax, M in enumerate(mats):
        y = np.moveaxis(np.tensordot(M, np.moveaxis(y, ax, 0), axes=(1, 0)), 0, ax)
    return y


def prolong(c):
    """I c: coarse correction -> fine; corrections vanish on the Dirichlet faces."""
    c = np.where(dirichlet_mask(c.shape), 0.0, c)
    f = _apply_axes(c, _axis_mats(_m_of(c.shape)))
    f[dirichlet_mask(f.shape)] = 0.0
    return f


def restrict(r):
    """R r = I^T r; Dirichlet entries are 0 on both grids."""
    r = np.where(dirichlet_mask(r.shape), 0.0, r)
    mc = _m_of(r.shape) // 2
    c = _apply_axes(r, [M.T for M in _axis_mats(mc)])
    c[dirichlet_mask(c.shape)] = 0.0
    return c


def project(x):
    """Projection of the iterate: I^T x with every row divided by its sum (2^3
    away from the free faces, the paper's 2^-d I^T there); injection of the
    Dirichlet data on the faces x = 0 and x = 10."""
    mc = _m_of(x.shape) // 2
    mats = [M.T for M in _axis_mats(mc)]
    c = _apply_axes(x, mats)
    rows = _apply_axes(np.ones(x.shape), mats)
    c = c / rows
    inj = x[::2, ::2, ::2, :]
    dm = dirichlet_mask(c.shape)
    c[dm] = inj[dm]
    return c
