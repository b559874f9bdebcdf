"""Pin of the oracle's adjoint gradient: central differences of the loss
1/2 ||u(kappa) - u_obs||^2 along seeded directions, each u(kappa) from an
exact-Newton solve, agree with -(dF/dkappa)^T lambda."""
import numpy as np

from oracle import adjoint, fem
from workloads import kappa_field, noise_like


def test_adjoint_gradient_matches_central_differences():
    n = 6
    kap = kappa_field(n, seed=5, m=8)
    kap_obs = kappa_field(n, seed=6, m=8)
    u0 = np.zeros((n + 1,) * 3)
    u_obs, _ = adjoint.newton_direct("ndk3d", u0, kappa=kap_obs)
    u_obs = u_obs + noise_like(u_obs, 0.01, seed=7)
    u, _ = adjoint.newton_direct("ndk3d", u0, kappa=kap)
    grad, lam = adjoint.adjoint_gradient(u, kap, u_obs)
    rng = np.random.default_rng(8)
    for _ in range(4):
        dk = kap * rng.standard_normal(kap.shape)
        t = 1e-5
        up, _ = adjoint.newton_direct("ndk3d", u, kappa=kap + t * dk)
        um, _ = adjoint.newton_direct("ndk3d", u, kappa=kap - t * dk)
        fd = (adjoint.loss(up, u_obs) - adjoint.loss(um, u_obs)) / (2 * t)
        an = float(np.sum(grad * dk))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_grf_kappa_statistics():
    """The coefficient field is exp of a zero-mean field with variance 0.5."""
    from workloads import grf_on_grid
    g = grf_on_grid(32, 0.1, 0.5, seed=5)
    assert abs(g.var() - 0.5) < 0.15 and abs(g.mean()) < 0.3
    k = kappa_field(16, seed=5)
    assert k.shape == (16, 16, 16) and np.all(k > 0)
