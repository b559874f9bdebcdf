"""Direct solves and the adjoint gradient (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

newton_direct: Newton's method x <- x - J(x)^-1 F(x) with the assembled analytic
    Jacobian and a sparse direct solve at every step (Sec. 1 with the linear
    system solved exactly).  The discrete solution of F(u) = 0 is unique for the
    problems it is used on here, so this reaches the same u as the Jacobian-free method
    by an independent route; it is the reference for final-solution parity.

adjoint_gradient: for the coefficient problem ndk3d and the loss
    1/2 ||u(kappa) - u_obs||^2 over interior nodes, solve J(u)^T lambda = u - u_obs
    with the assembled Jacobian and return grad_kappa = -(dF/dkappa)^T lambda
    (implicit-function theorem: F(u(kappa), kappa) = 0 gives
    du/dkappa = -J^-1 dF/dkappa).  The paper has no adjoint; this is the plain
    definition of the gradient of the stated loss.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import fem


def _interior_system(J, mask):
    idx = np.flatnonzero(mask.ravel())
    return J[idx][:, idx].tocsc(), idx


def newton_direct(kind, u0, lam=0.0, kappa=None, load=None, rtol=1e-13, max_it=30):
    """Exact Newton on the interior unknowns.  Returns (u, list of ||F||)."""
    u = u0.copy()
    mask = fem.interior(u.shape)
    F = fem.residual(kind, u, lam, kappa, load)
    F0 = np.linalg.norm(F[mask])
    hist = [F0]
    for _ in range(max_it):
        if hist[-1] <= rtol * F0 or hist[-1] == 0.0:
            break
        J = fem.assemble_jacobian(kind, u, lam, kappa)
        A, idx = _interior_system(J, mask)
        du = spla.spsolve(A, -F.ravel()[idx])
        uf = u.ravel().copy()
        uf[idx] += du
        u = uf.reshape(u.shape)
        F = fem.residual(kind, u, lam, kappa, load)
        hist.append(np.linalg.norm(F[mask]))
    return u, hist


def adjoint_gradient(u, kappa, u_obs):
    """(grad_kappa, lambda) for L = 1/2 ||u - u_obs||^2 (interior nodes) at a solution u."""
    mask = fem.interior(u.shape)
    g = np.where(mask, u - u_obs, 0.0)
    J = fem.assemble_jacobian("ndk3d", u, 0.0, kappa)
    A, idx = _interior_system(J, mask)
    lam_i = spla.spsolve(A.T.tocsc(), g.ravel()[idx])
    lam = np.zeros(u.size)
    lam[idx] = lam_i
    lam = lam.reshape(u.shape)
    _, dk = fem.vjp_ndk3d(u, kappa, lam)
    return -dk, lam


def loss(u, u_obs):
    """Misfit 1/2 ||u - u_obs||^2 over the interior nodes (the coefficient
    problem's loss; the paper has no adjoint)."""
    mask = fem.interior(u.shape)
    return 0.5 * float(np.sum((u[mask] - u_obs[mask]) ** 2))
