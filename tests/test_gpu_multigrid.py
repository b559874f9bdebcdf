"""GPU parity of the multigrid building blocks (Sec. 2, Alg. 1) and of the
JFNK solve (Sec. 1, Sec. 3) against the oracle, through the C ABI.

FD-driven components (power method, smoother, coarse GMRES, V-cycle) carry the
FD round-off of each action (about eps_p / eps relative, ~1e-8 for FP64), so
GPU and oracle agree to ~1e-6 relative, not to the last bit; transfers are
exact linear maps and agree to round-off."""
import functools

import numpy as np
import pytest

from gpu_common import dev, host, jf, kernel_path, rel, torch
from oracle import adjoint, fem, jfnk, transfer
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu


def _opts(**kw):
    return jf().default_options(**kw)


class _LinearLevel(jfnk.Level):
    """Oracle level whose F is the exact linearisation F(w) = J(x)(w - x), so the
    oracle's FD action becomes the exact J v (used to measure FD deviation)."""

    def __init__(self, lv):
        super().__init__(lv.kind, lv.n, lv.lam, lv.kappa, lv.load)
        self.x0 = lv.x
        self.J = fem.assemble_jacobian(lv.kind, lv.x, lv.lam, lv.kappa)

    def F(self, w):
        self.ge += 1
        return (self.J @ (w - self.x0).ravel()).reshape(w.shape)


def _fd_tol(oracle_fd, oracle_exact, floor=1e-10):
    """GPU and oracle each carry FD round-off and truncation of the same size;
    bound their difference by 3x the oracle's own deviation from the exact-J
    result (the FD error scale of this configuration)."""
    return max(floor, 3.0 * rel(oracle_fd, oracle_exact))


@pytest.mark.parametrize("d,n", [(2, 8), (2, 66), (3, 6), (3, 34)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_transfers_parity(d, n, dt):
    kind = "bratu2d" if d == 2 else "nd3d"
    p = jf().Problem(kind, n, 2, lam=1.0)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-14 if dt == "f64" else 1e-6
    xf = random_state_field(n, d, seed=3, kind="uniform")
    xf[fem.boundary_mask(xf.shape)] = 0.0
    xb = xf.copy()
    xb[fem.boundary_mask(xb.shape)] = 0.7   # Dirichlet data for the projection
    c = random_state_field(n // 2, d, seed=4, kind="uniform")
    r = host(p.transfer("restrict", dev(xf, tdt)))
    assert rel(r, transfer.restrict(xf)) <= tol
    pr = host(p.transfer("project", dev(xb, tdt)))
    assert rel(pr, transfer.project(xb)) <= tol
    s0 = random_state_field(n, d, seed=5, kind="uniform")
    out = dev(s0, tdt)
    p.transfer("prolong_add", dev(c, tdt), out=out)
    assert rel(host(out), s0 + transfer.prolong(c)) <= tol


@functools.lru_cache(maxsize=None)
def _oracle_setup(kind, n, levels, pc, seed, lam, nu_pre, nu_post, cheb_degree, power_iters, power_tol=0.0):
    """The oracle hierarchy after set-up at the seeded state (shared by the tests
    and kernel paths that use the same case; tests only read it, or set the
    fields they use before using them)."""
    d = fem.dim_of(kind)
    u = random_state_field(n, d, seed=9, kind="mms" if kind == "nd3d" else "uniform",
                           amplitude=0.1 if kind == "nd3d" else 0.5)
    load = fem.mms_load(n) if kind == "nd3d" else None
    lv = jfnk.build_hierarchy(kind, n, levels, lam=lam, load=load)
    oo = jfnk.Options(nu_pre=nu_pre, nu_post=nu_post, cheb_degree=cheb_degree, power_iters=power_iters,
                      power_tol=power_tol, eps_mode_pc="fp32" if pc == "f32" else "paper", seed=seed)
    jfnk.setup_levels(lv, u, oo, 0)
    return lv, oo, u, tuple(x.lam_max for x in lv)


def _setup_pair(kind, n, levels, pc="f64", seed=0, lam=5.0, **kw):
    """GPU problem after mg_setup at a seeded state, and the oracle hierarchy
    after the same set-up."""
    o = _opts(pc_dtype=jf().F32 if pc == "f32" else jf().F64,
              eps_mode_pc=jf().EPS_FP32 if pc == "f32" else jf().EPS_PAPER, seed=seed, **kw)
    p = jf().Problem(kind, n, levels, lam=lam, options=o)
    lv, oo, u, lam0 = _oracle_setup(kind, n, levels, pc, seed, lam, o.nu_pre, o.nu_post, o.cheb_degree,
                                    o.power_iters, o.power_tol)
    for x, lm in zip(lv, lam0):  # a test may have set the GPU's estimates
        x.lam_max = lm
    p.mg_setup(dev(u), 0)
    return p, o, lv, oo, u


@pytest.mark.parametrize("kind,n,levels", [("bratu2d", 64, 4), ("nd3d", 32, 4)])
@pytest.mark.parametrize("power", [(10, 0.0), (30, 1e-2)], ids=["fixed10", "rule"])
def test_setup_projection_operator_and_power_method(kind, n, levels, power):
    """Projection, A(x_l), the x statistics and the power method on every level.
    power: a fixed count, or the Sec. 2 rule (at most 30 iterations, stop when
    successive estimates differ by less than 1e-2 relative), where the library
    checks every level's estimate after each round of iterations."""
    p, o, lv, oo, u = _setup_pair(kind, n, levels, power_iters=power[0], power_tol=power[1])
    for l in range(levels):
        x = host(p.level_vector(l, "x"))
        assert rel(x, lv[l].x) <= 1e-14
        Ax = host(p.level_vector(l, "Ax"))
        A_ora = fem.operator(kind, lv[l].x, 5.0)
        assert rel(Ax, A_ora) <= 1e-12
        info = p.level_info(l)
        m = lv[l].mask
        assert info["sum_abs_x"] == pytest.approx(np.abs(lv[l].x[m]).sum(), rel=1e-12)
        if l >= 1:
            # same SplitMix64 start vector, the same FD power iterations on both sides
            assert info["lambda_max"] == pytest.approx(lv[l].lam_max, rel=1e-6), l
            # the eigenvector estimate is a direction: the library keeps the last
            # action's output J v/||v||, the oracle the normalised vector
            pv = host(p.level_vector(l, "power"))
            po = lv[l].power_v
            assert rel(pv / np.linalg.norm(pv), po / np.linalg.norm(po)) <= 1e-5


@pytest.mark.parametrize("kind,n,levels,path", [("bratu2d", 64, 4, "default"), ("nd3d", 32, 4, "default"),
                                                ("nd3d", 32, 4, "tiled"), ("nd3d", 32, 4, "zm"),
                                                ("nd3d", 64, 5, "default"), ("nd3d", 64, 5, "tiled"),
                                                ("nd3d", 64, 5, "zm")])
@pytest.mark.parametrize("nu,zero", [(1, True), (3, True), (2, False)])
def test_chebyshev_smoother_parity(kind, n, levels, path, nu, zero, monkeypatch):
    kernel_path(monkeypatch, path)
    p, o, lv, oo, u = _setup_pair(kind, n, levels)
    l = levels - 1
    d = fem.dim_of(kind)
    b = random_direction(n, d, seed=31) * 1e-3
    s0 = np.zeros_like(b) if zero else random_direction(n, d, seed=32) * 1e-3
    s = dev(s0)
    p.smooth(dev(b), s, level=l, nu=nu, s_is_zero=zero)
    lam = p.level_info(l)["lambda_max"]
    so = jfnk.chebyshev(lv[l], s0.copy(), lv[l].x, lv[l].Fx, b, nu, o.cheb_degree, lam, o.cheb_lo, o.cheb_hi)
    ll = _LinearLevel(lv[l])
    se = jfnk.chebyshev(ll, s0.copy(), lv[l].x, np.zeros_like(b), b, nu, o.cheb_degree, lam, o.cheb_lo, o.cheb_hi)
    assert rel(host(s), so) <= _fd_tol(so, se)


@pytest.mark.parametrize("n,levels,path", [(64, 5, p) for p in ("default", "tiled", "v2", "v3two", "v3mixed", "ep",
                                                                  "zm")]
                         + [(32, 4, p) for p in ("default", "ep", "zm", "cluster")])
def test_chebyshev_smoother_fp32_3d(n, levels, path, monkeypatch):
    """FP32 smoothing on the finest level of a 65^3 / 33^3 hierarchy (on the
    "tiled" path the two-elements-per-thread halo-free kernel, on "v2" the
    one-element kernel, on "ep"/"default" the element-parallel kernels, on
    "cluster" the one-cluster kernel): every fused Chebyshev mode against the
    oracle's FP64 smoother to FP32-FD accuracy, and the FP32 kernels against
    each other to the FP32 FD round-off."""
    kernel_path(monkeypatch, path)
    p, o, lv, oo, u = _setup_pair("nd3d", n, levels, pc="f32")
    l = levels - 1
    b = random_direction(n, 3, seed=31) * 1e-3
    s0 = random_direction(n, 3, seed=32) * 1e-3
    lam = p.level_info(l)["lambda_max"]
    for zero, nu in ((True, 1), (False, 2)):
        init = np.zeros_like(b) if zero else s0
        s = dev(init, torch.float32)
        p.smooth(dev(b, torch.float32), s, level=l, nu=nu, s_is_zero=zero)
        so = jfnk.chebyshev(lv[l], init.copy(), lv[l].x, lv[l].Fx, b, nu, o.cheb_degree, lam, o.cheb_lo,
                            o.cheb_hi, mode="fp32")
        assert rel(host(s), so) <= 1e-3
        _FP32_SMOOTH.setdefault((n, zero, nu), {})[path] = host(s)
    # every path run so far in this session agrees to the FP32 FD round-off:
    # each action carries ~2^-23 / sqrt(2^-23) = 3.5e-4 relative noise of its own
    # rounding order, of which 1e-3 leaves room for a few actions
    for runs in _FP32_SMOOTH.values():
        ref = next(iter(runs.values()))
        for other in runs.values():
            assert rel(other, ref) <= 1e-3


_FP32_SMOOTH = {}


@pytest.mark.parametrize("kind,n,levels", [("bratu2d", 64, 4), ("nd3d", 32, 4)])
def test_coarse_gmres_parity(kind, n, levels):
    p, o, lv, oo, u = _setup_pair(kind, n, levels)
    d = fem.dim_of(kind)
    n0 = n >> (levels - 1)
    b = random_direction(n0, d, seed=41)
    s = host(p.coarse_solve(dev(b)))
    lv0 = lv[0]
    so, its, _ = jfnk.gmres(lambda v: jfnk.fd_jv(lv0, lv0.x, lv0.Fx, v), b, lv0.mask, 1e-12, lv0.n_unknowns)
    ll = _LinearLevel(lv0)
    se, _, _ = jfnk.gmres(lambda v: jfnk.fd_jv(ll, lv0.x, np.zeros_like(b), v), b, lv0.mask, 1e-12, lv0.n_unknowns)
    assert rel(s, so) <= _fd_tol(so, se, 1e-9)


@pytest.mark.parametrize("kind,n,levels,path", [("bratu2d", 64, 4, "default"), ("nd3d", 32, 4, "default"),
                                                ("nd3d", 16, 2, "default"), ("nd3d", 64, 5, "default"),
                                                ("nd3d", 64, 5, "tiled"), ("nd3d", 64, 5, "zm")])
def test_vcycle_parity(kind, n, levels, path, monkeypatch):
    """One V-cycle of Alg. 1 with the GPU's lambda_l given to the oracle."""
    kernel_path(monkeypatch, path)
    kw = dict(nu_pre=2, nu_post=2, cheb_degree=4) if kind == "nd3d" else {}
    p, o, lv, oo, u = _setup_pair(kind, n, levels, **kw)
    for l in range(1, levels):
        lv[l].lam_max = p.level_info(l)["lambda_max"]
    b = random_direction(n, fem.dim_of(kind), seed=51)
    s = host(p.mg_vcycle(dev(b)))
    so = jfnk.mg_vcycle(lv, levels - 1, b, oo)
    lin = []
    for x in lv:
        ll = _LinearLevel(x)
        ll.x, ll.Fx, ll.lam_max = x.x, np.zeros(x.shape), x.lam_max
        lin.append(ll)
    se = jfnk.mg_vcycle(lin, levels - 1, b, oo)
    assert rel(s, so) <= _fd_tol(so, se, 1e-9)


@pytest.mark.parametrize("kind,n,levels,path", [("bratu2d", 64, 4, "default"), ("nd3d", 32, 4, "ep"),
                                                ("nd3d", 32, 4, "cluster")])
@pytest.mark.parametrize("pc", ["f64", "f32"])
def test_vcycle_fp32_parity_and_contraction(pc, kind, n, levels, path, monkeypatch):
    """The FP32 preconditioner agrees with the FP64 oracle to FP32 accuracy."""
    kernel_path(monkeypatch, path)
    p, o, lv, oo, u = _setup_pair(kind, n, levels, pc=pc)
    for l in range(1, levels):
        lv[l].lam_max = p.level_info(l)["lambda_max"]
    b = random_direction(n, fem.dim_of(kind), seed=61)
    bd = dev(b, torch.float64)
    s = host(p.mg_vcycle(bd))
    so = jfnk.mg_vcycle(lv, levels - 1, b, oo)
    assert rel(s, so) <= (1e-6 if pc == "f64" else 1e-3)


@pytest.mark.parametrize("pc", ["f64", "f32"])
def test_solve_bratu_matches_discrete_solution(pc):
    """Bratu lambda = 5 on 65x65 nodes, 4 levels, V(3,3) degree 3, FGMRES(30),
    rtol 1e-10: the GPU solution equals the exact-Newton discrete solution."""
    n = 64
    o = _opts(rtol_newton=1e-11, pc_dtype=jf().F32 if pc == "f32" else jf().F64,
              eps_mode_pc=jf().EPS_FP32 if pc == "f32" else jf().EPS_PAPER)
    p = jf().Problem("bratu2d", n, 4, lam=5.0, options=o)
    u = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
    st = p.solve(u)
    ud, _ = adjoint.newton_direct("bratu2d", np.zeros((n + 1, n + 1)), lam=5.0)
    assert st["converged"]
    assert rel(host(u), ud) <= 1e-8
    assert st["newton_its"] <= 6


@functools.lru_cache(maxsize=None)
def _nd_direct_solution(n):
    return adjoint.newton_direct("nd3d", np.zeros((n + 1,) * 3), load=fem.mms_load(n))[0]


@pytest.mark.parametrize("pc,path", [("f64", "default"), ("f32", "default"), ("f64", "tiled"), ("f32", "ep"),
                                     ("f64", "zm"), ("f32", "zm"), ("f32", "cluster")])
def test_solve_nd_matches_discrete_solution(pc, path, monkeypatch):
    kernel_path(monkeypatch, path)
    n = 24  # 25^3 nodes, 4 levels down to 3^3 elements (a sparse direct solve at this size is quick)
    o = _opts(rtol_newton=1e-11, nu_pre=2, nu_post=2, cheb_degree=4,
              pc_dtype=jf().F32 if pc == "f32" else jf().F64,
              eps_mode_pc=jf().EPS_FP32 if pc == "f32" else jf().EPS_PAPER)
    p = jf().Problem("nd3d", n, 4, options=o)
    u = torch.zeros((n + 1,) * 3, dtype=torch.float64, device="cuda")
    st = p.solve(u)
    ud = _nd_direct_solution(n)
    assert st["converged"]
    assert rel(host(u), ud) <= 1e-8


@pytest.mark.parametrize("kind,n,levels,path", [("bratu2d", 64, 4, "default"), ("nd3d", 32, 4, "default"),
                                                ("nd3d", 32, 4, "cluster")])
def test_graph_replay_matches_direct_launches(kind, n, levels, path, monkeypatch):
    """The V-cycle replayed from a captured CUDA graph runs the same kernels on
    the same device scalars: the solve is bit-identical to direct launches."""
    kernel_path(monkeypatch, path)
    d = fem.dim_of(kind)
    sols, stats = [], []
    for g in (0, 1):
        o = _opts(use_graph=g, pc_dtype=jf().F32, eps_mode_pc=jf().EPS_FP32)
        p = jf().Problem(kind, n, levels, lam=5.0, options=o)
        u = torch.zeros((n + 1,) * d, dtype=torch.float64, device="cuda")
        stats.append(p.solve(u))
        sols.append(host(u))
    assert np.array_equal(sols[0], sols[1])
    assert stats[0]["linear_its"] == stats[1]["linear_its"] and stats[0]["ge"] == stats[1]["ge"]
