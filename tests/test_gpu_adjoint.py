"""GPU parity of the adjoint path (vector-Jacobian products, adjoint solve,
autograd) against the oracle and against central differences of the loss
1/2 ||u(kappa) - u_obs||^2 through GPU forward solves."""
import functools

import numpy as np
import pytest

from gpu_common import dev, host, jf, kernel_path, rel, torch
from oracle import adjoint, fem
from workloads import kappa_field, noise_like, random_direction, random_state_field

pytestmark = pytest.mark.gpu


def _opts(pc="f64", rtol=1e-11):
    m = jf()
    return m.default_options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=rtol,
                             pc_dtype=m.F32 if pc == "f32" else m.F64,
                             eps_mode_pc=m.EPS_FP32 if pc == "f32" else m.EPS_PAPER)


@functools.lru_cache(maxsize=None)
def _oracle_vjp_case(kind, n):
    """Inputs and the oracle's J^T w and (dF/dkappa)^T w of one case, shared by
    the precisions and kernel paths."""
    kap = np.exp(np.random.default_rng(2).normal(size=(n, n, n))) if kind == "ndk3d" else None
    u = random_state_field(n, 3, seed=4, amplitude=0.7)
    u[fem.boundary_mask(u.shape)] = 0.2
    w = random_direction(n, 3, seed=5)
    w[fem.boundary_mask(w.shape)] = 0.9  # boundary entries of w are not equations: ignored
    J0, d0 = fem.vjp_ndk3d(u, kap if kap is not None else np.ones((n, n, n)), w)
    JaT = None
    if n <= 20:  # the transpose of the assembled analytic Jacobian, independently
        Ja = fem.assemble_jacobian("ndk3d", u, 0.0, kap if kap is not None else np.ones((n, n, n)))
        wm = np.where(fem.interior(u.shape), w, 0.0)
        JaT = (Ja.T @ wm.ravel()).reshape(u.shape)
    return u, w, kap, J0, d0, JaT


@pytest.mark.parametrize("kind,n", [("ndk3d", 5), ("ndk3d", 20), ("ndk3d", 37), ("nd3d", 33), ("ndk3d", 64)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("path", ["default", "ep", "tiled"])
def test_vjp_parity(kind, n, dt, path, monkeypatch):
    kernel_path(monkeypatch, path)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-12 if dt == "f64" else 1e-5
    u, w, kap, J0, d0, JaT = _oracle_vjp_case(kind, n)
    p = jf().Problem(kind, n, 1, kappa=None if kap is None else torch.as_tensor(kap))
    if kind == "ndk3d":
        JTw, dk = p.vjp(dev(u, tdt), dev(w, tdt), dkappa=True)
        assert rel(host(dk), d0) <= tol
    else:
        JTw = p.vjp(dev(u, tdt), dev(w, tdt))
    assert rel(host(JTw), J0) <= tol
    if dt == "f64" and JaT is not None:
        assert rel(host(JTw), JaT) <= 1e-12


@functools.lru_cache(maxsize=None)
def _observations(n):
    """kappa, and u_obs from the second coefficient field plus 1 % noise."""
    kap = kappa_field(n, seed=5)
    kap2 = kappa_field(n, seed=6)
    u_obs, _ = adjoint.newton_direct("ndk3d", np.zeros((n + 1,) * 3), kappa=kap2)
    return kap, u_obs + noise_like(u_obs, 0.01, seed=7)


@functools.lru_cache(maxsize=None)
def _oracle_adjoint(n):
    """The oracle's forward solution, adjoint and gradient (exact Newton, sparse
    direct adjoint solve), shared by the precisions and kernel paths."""
    kap, u_obs = _observations(n)
    u_ora, _ = adjoint.newton_direct("ndk3d", np.zeros((n + 1,) * 3), kappa=kap)
    grad_ora, lam_ora = adjoint.adjoint_gradient(u_ora, kap, u_obs)
    return u_ora, grad_ora, lam_ora


def _adjoint_case(n, levels, pc="f64"):
    kap, u_obs = _observations(n)
    o = _opts(pc)
    p = jf().Problem("ndk3d", n, levels, kappa=torch.as_tensor(kap), options=o)
    return p, o, kap, u_obs


@pytest.mark.parametrize("pc,path", [("f64", "default"), ("f32", "default"), ("f64", "tiled")])
def test_adjoint_solve_matches_oracle_adjoint(pc, path, monkeypatch):
    """At 33^3 nodes: the multigrid-preconditioned GPU adjoint agrees with the
    oracle's adjoint (assembled J^T, sparse direct solve) to 1e-8."""
    kernel_path(monkeypatch, path)
    n = 32
    p, o, kap, u_obs = _adjoint_case(n, 4, pc)
    u = torch.zeros((n + 1,) * 3, dtype=torch.float64, device="cuda")
    st = p.solve(u)
    assert st["converged"]
    g = u - dev(u_obs)
    lam, gk, ast = p.adjoint_solve(u, g, rtol=1e-12)
    u_ora, grad_ora, lam_ora = _oracle_adjoint(n)
    assert rel(host(u), u_ora) <= 1e-8
    assert rel(host(lam), lam_ora) <= 1e-8
    assert rel(host(gk), grad_ora) <= 1e-8
    assert ast["linear_its"] <= 60


@pytest.mark.parametrize("n,levels,ndir", [(32, 4, 6), (128, 6, 16)])
def test_gradient_matches_central_differences(n, levels, ndir):
    """Central differences of the loss along seeded directions dkappa = kappa * z,
    each loss from a GPU forward solve, against grad_kappa . dkappa (16
    directions at 129^3 nodes, the size of the coefficient workload)."""
    kap = kappa_field(n, seed=5)
    kap2 = kappa_field(n, seed=6)
    o = _opts("f64", rtol=1e-11)
    p = jf().Problem("ndk3d", n, levels, kappa=torch.as_tensor(kap), options=o)
    mask = torch.as_tensor(fem.interior((n + 1,) * 3)).cuda()

    def solve(k):
        p.set_kappa(torch.as_tensor(k))
        u = torch.zeros((n + 1,) * 3, dtype=torch.float64, device="cuda")
        p.solve(u)
        return u

    u_obs = solve(kap2)
    u_obs = u_obs + dev(noise_like(host(u_obs), 0.01, seed=7))
    u = solve(kap)
    loss = lambda uu: 0.5 * float(((uu - u_obs)[mask] ** 2).sum())
    _, gk, _ = p.adjoint_solve(u, u - u_obs, rtol=1e-12)
    gk = host(gk)
    rng = np.random.default_rng(8)
    # L(k+) - L(k-) = 1/2 (u+ - u-) . (u+ + u- - 2 u_obs) avoids the cancellation of
    # subtracting two losses; t balances the O(t^2) truncation of the central
    # difference against the forward-solve error divided by t (~1e-6 each)
    t = 3e-4
    for _ in range(ndir):
        dk = kap * rng.standard_normal(kap.shape)
        up, um = solve(kap + t * dk), solve(kap - t * dk)
        fd = 0.5 * float(((up - um) * (up + um - 2 * u_obs))[mask].sum()) / (2 * t)
        an = float(np.sum(gk * dk))
        assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)


def test_autograd_function_backward():
    from paper_2103_13890_gb300.autograd import JFNKSolve
    n = 16
    p, o, kap, u_obs = _adjoint_case(n, 3)
    kt = torch.tensor(kap, device="cuda", requires_grad=True)
    u = JFNKSolve.apply(kt, p)
    mask = torch.as_tensor(fem.interior((n + 1,) * 3)).cuda()
    loss = 0.5 * ((u - dev(u_obs))[mask] ** 2).sum()
    loss.backward()
    u_ora, _ = adjoint.newton_direct("ndk3d", np.zeros((n + 1,) * 3), kappa=kap)
    grad_ora, _ = adjoint.adjoint_gradient(u_ora, kap, u_obs)
    assert rel(host(kt.grad), grad_ora) <= 1e-8
