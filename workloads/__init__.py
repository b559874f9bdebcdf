"""Seeded synthetic inputs shaped like the solver's target workloads (listed below).

This module is the only code shared by the oracle side (tests, CPU baseline)
and the CUDA side (tests, bench).  It holds none of the method's arithmetic:
no residual, no Jacobian action, no transfer, no solver step.  It only draws
seeded random fields, coefficient fields and instance parameters.

Workloads (all inputs analytic or seeded; the paper's own examples are analytic,
Sec. 3, so no dataset is stood in for):
  bratu65     2D Bratu, lambda = 5, 65x65 nodes (64 elements), 4 levels, u0 = 0
  nd129       3D nonlinear diffusion, manufactured u*, 129^3 nodes, 6 levels, u0 = 0
  nd257       same at 257^3 nodes, 7 levels
  batch64     64 Bratu instances, sizes from {129^2, 257^2, 513^2}, lambda ~ U[1, 6.5]
  adjoint129  3D coefficient problem, 129^3 nodes, kappa = exp(g), g a Gaussian
              random field (squared-exponential covariance, length 0.1,
              variance 0.5, sampled on 32^3 nodes, trilinearly interpolated to
              element centres)
"""
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "random_state_field", "random_direction",
    "batch_instances", "grf_on_grid", "kappa_field", "noise_like",
]


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "bratu2d" | "nd3d" | "ndk3d"
    n: int             # elements per direction on the finest level
    levels: int
    lam: float = 0.0
    nu_pre: int = 3
    nu_post: int = 3
    cheb_degree: int = 3
    rtol: float = 1e-8


WORKLOADS = {
    "bratu65": Workload("bratu65", "bratu2d", 64, 4, lam=5.0, nu_pre=3, nu_post=3, cheb_degree=3, rtol=1e-10),
    "nd129": Workload("nd129", "nd3d", 128, 6, nu_pre=2, nu_post=2, cheb_degree=4, rtol=1e-8),
    "nd257": Workload("nd257", "nd3d", 256, 7, nu_pre=2, nu_post=2, cheb_degree=4, rtol=1e-8),
    "adjoint129": Workload("adjoint129", "ndk3d", 128, 6, nu_pre=2, nu_post=2, cheb_degree=4, rtol=1e-8),
}


def _boundary_zero(a):
    for ax in range(a.ndim):
        sl = [slice(None)] * a.ndim
        sl[ax] = 0
        a[tuple(sl)] = 0.0
        sl[ax] = -1
        a[tuple(sl)] = 0.0
    return a


def random_state_field(n, d, seed, kind="uniform", amplitude=1.0):
    """A seeded nodal field on (n+1)^d nodes with zero boundary values.
    kind="uniform": U(-amplitude, amplitude) on interior nodes.
    kind="mms":     sin(pi x) sin(pi y) sin(pi z) + amplitude * N(0,1) (3D only)."""
    rng = np.random.default_rng(seed)
    shape = (n + 1,) * d
    if kind == "uniform":
        a = rng.uniform(-amplitude, amplitude, size=shape)
    elif kind == "mms":
        t = np.linspace(0.0, 1.0, n + 1)
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        a = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) + amplitude * rng.standard_normal(shape)
    else:
        raise ValueError(kind)
    return _boundary_zero(a)


def random_direction(n, d, seed):
    """A seeded N(0,1) direction on interior nodes (boundary zero)."""
    rng = np.random.default_rng(seed)
    return _boundary_zero(rng.standard_normal((n + 1,) * d))


def batch_instances(count=64, seed=4, sizes=(128, 256, 512), lam_range=(1.0, 6.5)):
    """(n_elements, lambda) for each instance of the batched Bratu workload."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    lams = rng.uniform(lam_range[0], lam_range[1], size=count)
    return [(int(a), float(b)) for a, b in zip(ns, lams)]


def grf_on_grid(m=32, length=0.1, variance=0.5, seed=5):
    """Gaussian random field on the m^3 nodes linspace(0,1,m)^3 with covariance
    variance * exp(-|x-y|^2 / (2 length^2)), sampled separably: the covariance is
    a Kronecker product of three 1D kernels, each factored by its
    eigendecomposition (negative round-off eigenvalues clipped to 0)."""
    t = np.linspace(0.0, 1.0, m)
    K1 = np.exp(-((t[:, None] - t[None, :]) ** 2) / (2.0 * length ** 2))
    w, V = np.linalg.eigh(K1)
    L1 = V * np.sqrt(np.clip(w, 0.0, None))[None, :]
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((m, m, m))
    g = np.einsum("ai,bj,ck,ijk->abc", L1, L1, L1, z, optimize=True)
    return np.sqrt(variance) * g


def kappa_field(n, seed=5, m=32, length=0.1, variance=0.5):
    """Per-element kappa = exp(g) on an n^3 element grid, g trilinearly
    interpolated from the m^3 random field to element centres (i + 1/2)/n."""
    g = grf_on_grid(m, length, variance, seed)
    c = (np.arange(n) + 0.5) / n * (m - 1)
    i0 = np.clip(np.floor(c).astype(int), 0, m - 2)
    f = c - i0
    gz = g[i0] * (1 - f)[:, None, None] + g[i0 + 1] * f[:, None, None]
    gy = gz[:, i0] * (1 - f)[None, :, None] + gz[:, i0 + 1] * f[None, :, None]
    gx = gy[:, :, i0] * (1 - f)[None, None, :] + gy[:, :, i0 + 1] * f[None, None, :]
    return np.exp(gx)


def noise_like(a, rel, seed):
    """rel * RMS(a) * N(0,1) noise of a's shape (boundary zero)."""
    rng = np.random.default_rng(seed)
    rms = float(np.sqrt(np.mean(a * a)))
    return _boundary_zero(rel * rms * rng.standard_normal(a.shape))
