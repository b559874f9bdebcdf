"""GPU parity of the residual F(u) and the FD Jacobian action (Sec. 1) against
the oracle, element by element, through the C ABI.

Tolerances: F <= 1e-12 relative (FP64) and <= 1e-5 (FP32) at seeded random
states.  The FD action amplifies rounding of F(u + eps v) by 1/eps: two
correct FP64 implementations differ by about c eps_p ||F-terms|| / (eps ||Jv||);
the test computes that bound from the data (c = 64) rather than fixing it."""
import functools

import numpy as np
import pytest

from gpu_common import dev, host, jf, kernel_path, rel, torch
from oracle import fem, jfnk
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52


def _state(kind, n, seed, dirichlet=0.0):
    d = fem.dim_of(kind)
    u = random_state_field(n, d, seed=seed, kind="mms" if kind == "nd3d" else "uniform",
                           amplitude=0.1 if kind == "nd3d" else 0.9)
    if dirichlet:
        u[fem.boundary_mask(u.shape)] = dirichlet
    return u


def _problem(kind, n, levels=1, lam=5.0, kappa=None, options=None):
    return jf().Problem(kind, n, levels, lam=lam, kappa=None if kappa is None else torch.as_tensor(kappa),
                        options=options)


def _kappa(n, seed=3):
    return np.exp(np.random.default_rng(seed).normal(size=(n, n, n)))


# sizes span several 31 x 7 (3D) / row-segment (2D) tiles with ragged tails
# (3D grids with n a multiple of 32 and n >= 64 take the halo-free kernel with
# its face fixup, the others the tiled kernel, unless the element-parallel
# kernels run: "path" selects)
CASES = [("bratu2d", 7), ("bratu2d", 64), ("bratu2d", 95), ("bratu2d", 600),
         ("nd3d", 4), ("nd3d", 33), ("nd3d", 40), ("ndk3d", 5), ("ndk3d", 37),
         ("nd3d", 64), ("nd3d", 96), ("ndk3d", 64)]
PATH_CASES = [(k, n, path) for k, n in CASES for path in ("default", "ep", "zm", "tiled")
              if k != "bratu2d" or path == "default"]
# the FP32 one-element-per-thread halo-free kernel (the default FP32 kernel on
# these grids evaluates two elements per thread, CTAs per SM chosen per mode),
# the paired kernel with one or two CTAs per SM in every mode, and the 129^3
# grid in FP32
PATH_CASES += [(k, n, path) for k, n in CASES for path in ("v2", "v3one", "v3two")
               if k != "bratu2d" and n % 32 == 0 and n >= 64]
PATH_CASES += [("nd3d", 128, "default")]
# FP32 levels in one thread-block cluster: whole slices a CTA (n = 4, 16), two
# slices a CTA (32), a ragged last CTA (n = 5: 5 CTAs; 13; 27: 14 CTAs, the last
# with one slice)
PATH_CASES += [(k, n, "cluster") for k, n in (("nd3d", 4), ("ndk3d", 5), ("ndk3d", 13), ("nd3d", 16),
                                               ("nd3d", 27), ("nd3d", 32))]


@functools.lru_cache(maxsize=None)
def _oracle_residual_case(kind, n, dirichlet):
    """(u, kappa, oracle F) of one parity case, shared by the kernel paths."""
    kap = _kappa(n) if kind == "ndk3d" else None
    u = _state(kind, n, seed=n, dirichlet=dirichlet)
    load = fem.mms_load(n) if kind == "nd3d" else None
    return u, kap, fem.residual(kind, u, 5.0, kap, load)


@pytest.mark.parametrize("kind,n,path", PATH_CASES)
@pytest.mark.parametrize("dirichlet", [0.0, 0.3])
def test_residual_fp64_fp32_parity(kind, n, path, dirichlet, monkeypatch):
    kernel_path(monkeypatch, path)
    u, kap, F_ora = _oracle_residual_case(kind, n, dirichlet)
    p = _problem(kind, n, kappa=kap)
    F64 = host(p.residual(dev(u)))
    assert rel(F64, F_ora) <= 1e-12
    assert np.all(F64[fem.boundary_mask(u.shape)] == 0)
    F32 = host(p.residual(dev(u, torch.float32)))
    assert rel(F32, F_ora) <= 1e-5


@pytest.mark.parametrize("kind,n,path", [("bratu2d", 512, "default"), ("nd3d", 128, "default"),
                                         ("nd3d", 128, "tiled"), ("nd3d", 128, "ep"), ("nd3d", 256, "default"),
                                         ("ndk3d", 128, "default")])
def test_residual_full_size_sampled(kind, n, path, monkeypatch):
    """At the full workload sizes: the oracle evaluates F at 60 sampled nodes
    (its own element routine on the 2^d elements around each)."""
    kernel_path(monkeypatch, path)
    kap = _kappa(n) if kind == "ndk3d" else None
    p = _problem(kind, n, kappa=kap)
    u = _state(kind, n, seed=7)
    F = host(p.residual(dev(u)))
    rng = np.random.default_rng(1)
    nodes = [tuple(rng.integers(1, n, size=fem.dim_of(kind))) for _ in range(60)]
    nodes += [tuple([1] * fem.dim_of(kind)), tuple([n - 1] * fem.dim_of(kind))]
    Fs = fem.residual_at(kind, u, nodes, 5.0, kap, None)
    if kind == "nd3d":
        Fs = Fs - fem.mms_load_at(n, nodes)
    got = np.array([F[nd] for nd in nodes])
    scale = np.max(np.abs(Fs))
    assert np.max(np.abs(got - Fs)) <= 1e-12 * scale


def _fd_bound(kind, u, v, kap, load, eps):
    """c eps_p || |F terms| || / eps: round-off bound of the FD quotient."""
    d = fem.dim_of(kind)
    # magnitude of the summed terms: operator applied to |u| plus the load
    A_abs = np.abs(fem.operator(kind, np.abs(u), 5.0, kap))
    if load is not None:
        A_abs = A_abs + np.abs(load)
    return 64 * EPS64 * np.linalg.norm(A_abs) * 2 ** d / eps


@functools.lru_cache(maxsize=None)
def _oracle_jvp_case(kind, n):
    """Inputs, oracle FD action, its round-off bound and the analytic J v of one
    case, shared by the kernel paths."""
    kap = _kappa(n) if kind == "ndk3d" else None
    load = fem.mms_load(n) if kind == "nd3d" else None
    u = _state(kind, n, seed=11)
    v = random_direction(n, fem.dim_of(kind), seed=12)
    lv = jfnk.Level(kind, n, 5.0, kap, load)
    Fo = lv.F(u)
    eps = jfnk.fd_eps(u, v, lv.mask, "paper")
    Jo = jfnk.fd_jv(lv, u, Fo, v, "paper")
    bound = _fd_bound(kind, u, v, kap, load, eps) / np.linalg.norm(Jo)
    Jex = (fem.assemble_jacobian(kind, u, 5.0, kap) @ v.ravel()).reshape(u.shape)
    return u, v, kap, Jo, bound, Jex


@pytest.mark.parametrize("kind,n,path", [("bratu2d", 64, "default"), ("bratu2d", 95, "default"),
                                         ("nd3d", 33, "default"), ("nd3d", 33, "tiled"), ("nd3d", 33, "zm"),
                                         ("ndk3d", 20, "default"), ("ndk3d", 20, "tiled"), ("ndk3d", 20, "zm"),
                                         ("nd3d", 64, "default"), ("nd3d", 64, "tiled"), ("nd3d", 96, "default")])
def test_jvp_fp64_parity(kind, n, path, monkeypatch):
    kernel_path(monkeypatch, path)
    u, v, kap, Jo, bound, Jex = _oracle_jvp_case(kind, n)
    p = _problem(kind, n, kappa=kap)
    ud, vd = dev(u), dev(v)
    Fu = p.residual(ud)
    Jv = host(p.jvp(ud, Fu, vd))
    err = rel(Jv, Jo)
    assert err <= max(bound, 1e-12), (err, bound)
    # and both approximate the analytic action to FD accuracy
    assert rel(Jv, Jex) <= 1e-5


@pytest.mark.parametrize("kind,n,path", [("bratu2d", 64, "default"), ("nd3d", 33, "default"),
                                         ("nd3d", 33, "tiled"), ("nd3d", 33, "zm"), ("nd3d", 64, "default"),
                                         ("nd3d", 64, "ep"),
                                         ("nd3d", 64, "tiled"), ("nd3d", 64, "v2"), ("nd3d", 96, "default"),
                                         ("nd3d", 16, "cluster"), ("nd3d", 27, "cluster"),
                                         ("nd3d", 32, "cluster")])
def test_jvp_fp32_parity(kind, n, path, monkeypatch):
    """FP32 action with the single-precision step eps = sqrt(2^-23)(1+||u||)/||v||
    against the oracle's FP64 evaluation of the same quotient."""
    kernel_path(monkeypatch, path)
    load = fem.mms_load(n) if kind == "nd3d" else None
    p = _problem(kind, n)
    u = _state(kind, n, seed=21)
    v = random_direction(n, fem.dim_of(kind), seed=22)
    ud, vd = dev(u, torch.float32), dev(v, torch.float32)
    Fu = p.residual(ud)
    Jv = host(p.jvp(ud, Fu, vd, eps_mode=jf().EPS_FP32))
    lv = jfnk.Level(kind, n, 5.0, None, load)
    Jo = jfnk.fd_jv(lv, u, lv.F(u), v, "fp32")
    # the stated FP32 Jv tolerance; the kernels measure 1.6e-4 to 2e-4 here
    # (FP32 rounding of F(u + eps v) and F(u), 2^-23 each, over the step
    # eps ~ sqrt(2^-23) (1 + ||u||) / ||v||)
    assert rel(Jv, Jo) <= 1e-3


def test_jvp_explicit_eps_and_zero_direction():
    n = 16
    p = _problem("nd3d", n)
    u = _state("nd3d", n, seed=2)
    v = random_direction(n, 3, seed=3)
    ud, vd = dev(u), dev(v)
    Fu = p.residual(ud)
    Jv = host(p.jvp(ud, Fu, vd, eps=1e-7))
    lv = jfnk.Level("nd3d", n, 0.0, None, fem.mms_load(n))
    Jo = jfnk.fd_jv(lv, u, lv.F(u), v, eps=1e-7)
    assert rel(Jv, Jo) <= 1e-6
    Jz = host(p.jvp(ud, Fu, torch.zeros_like(vd)))
    assert np.all(Jz == 0)


@pytest.mark.parametrize("n,path", [(40, "default"), (128, "default"), (128, "tiled")])
def test_residual_deterministic(n, path, monkeypatch):
    kernel_path(monkeypatch, path)
    p = _problem("nd3d", n)
    ud = dev(_state("nd3d", n, seed=5))
    a = host(p.residual(ud))
    b = host(p.residual(ud))
    assert np.array_equal(a, b)
