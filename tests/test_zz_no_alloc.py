"""jfnk_jvp_noalloc, the FD Jacobian action for callers that cannot allocate
device memory (no problem object, no workspace; its scratch is a fixed array
inside libjfnk.so), gives the same result as jfnk_jvp, call after call.

This file is collected last so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process (the first
call on the device looks the scratch up) and after the other tests.  It also
compares the action with the oracle's FD quotient."""
import numpy as np
import pytest

from gpu_common import dev, host, jf, kernel_path, rel, torch
from oracle import fem, jfnk
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps_mode", ["paper", "fp32"])
@pytest.mark.parametrize("kind,n,dtype", [("nd3d", 33, "f64"), ("ndk3d", 20, "f64"), ("bratu2d", 95, "f32"),
                                          ("nd3d", 40, "f32")])
def test_jvp_noalloc_matches_jvp_on_two_calls_in_a_row(kind, n, dtype, eps_mode, monkeypatch):
    # the no-alloc entry runs the tiled kernel (it has no element scratch); the
    # problem object is made to run the same kernel, so both sum identically
    kernel_path(monkeypatch, "tiled")
    d = fem.dim_of(kind)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 1e-5
    kappa = np.exp(np.random.default_rng(3).normal(size=(n,) * d)) if kind == "ndk3d" else None
    load = fem.mms_load(n) if kind == "nd3d" else None
    p = jf().Problem(kind, n, 1, lam=5.0, load=None if load is None else torch.as_tensor(load),
                     kappa=None if kappa is None else torch.as_tensor(kappa))
    u = random_state_field(n, d, seed=n, kind="mms" if kind == "nd3d" else "uniform",
                           amplitude=0.1 if kind == "nd3d" else 0.8)
    ud = dev(u, tdt)
    Fu = p.residual(ud)
    kd = None if kappa is None else dev(kappa, tdt)
    ld = None if load is None else dev(load, tdt)
    mode = jf().EPS_PAPER if eps_mode == "paper" else jf().EPS_FP32
    for call in range(2):
        v = random_direction(n, d, seed=100 + call)
        vd = dev(v, tdt)
        ref = host(p.jvp(ud, Fu, vd, eps_mode=mode))
        got = host(jf().jvp_noalloc(kind, ud, Fu, vd, lam=5.0, kappa=kd, load=ld, eps_mode=mode))
        assert rel(got, ref) <= tol, (call, rel(got, ref))
        # an explicit FD step takes the other path through the scratch
        ref_e = host(p.jvp(ud, Fu, vd, eps=3e-7))
        got_e = host(jf().jvp_noalloc(kind, ud, Fu, vd, lam=5.0, kappa=kd, load=ld, eps=3e-7))
        assert rel(got_e, ref_e) <= tol


def test_jvp_noalloc_rejects_sizes_beyond_its_scratch():
    u = torch.zeros((3, 3, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(jf().JFNKError, match="INVALID_ARG"):
        jf().lib()  # library loaded
        import ctypes
        st = jf().lib().jfnk_jvp_noalloc(jf().ND3D, 1024, 0.0, None, None, jf().F64, ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), 0.0, 0, None)
        jf()._check(st)


@pytest.mark.parametrize("dtype,eps_mode", [("f64", "paper"), ("f64", "fp32"), ("f32", "fp32")])
def test_jvp_noalloc_matches_the_oracle(dtype, eps_mode):
    """The same action against the oracle's FD quotient (Sec. 1) evaluated in
    FP64 on the same inputs.  FP64: the two differ by the FD round-off of each
    side, which the test bounds from the data as the residual tests do:
    c eps_p ||(|A| |u| + |load|)|| 2^d / (eps ||Jv||) with c = 64 (a few 1e-7
    here with the paper's step; smaller with the single-precision step).  FP32
    (with the single-precision step, the one meant for FP32 vectors): the FP32
    round-off of the two residuals divided by the step, 2^-23 / sqrt(2^-23) ~
    3.5e-4 relative per evaluation; 1e-3 is the stated FP32 Jv tolerance
    (measured 1.6e-4 to 2e-4 on these kernels)."""
    kind, n, d = "nd3d", 24, 3
    load = fem.mms_load(n)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = random_state_field(n, d, seed=7, kind="mms", amplitude=0.1)
    v = random_direction(n, d, seed=8)
    if dtype == "f32":  # the oracle sees the inputs the kernel sees
        u = u.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
        load = load.astype(np.float32).astype(np.float64)
    lv = jfnk.Level(kind, n, 0.0, None, load)
    Fo = lv.F(u)
    Jo = jfnk.fd_jv(lv, u, Fo, v, eps_mode)
    mode = jf().EPS_PAPER if eps_mode == "paper" else jf().EPS_FP32
    ud, vd, ld, Fd = dev(u, tdt), dev(v, tdt), dev(load, tdt), dev(Fo, tdt)
    eps = jfnk.fd_eps(u, v, lv.mask, eps_mode)
    A_abs = np.abs(fem.operator(kind, np.abs(u))) + np.abs(load)
    bound = 64 * 2.0 ** -52 * np.linalg.norm(A_abs) * 2 ** d / eps / np.linalg.norm(Jo)
    for _ in range(2):
        got = host(jf().jvp_noalloc(kind, ud, Fd, vd, load=ld, eps_mode=mode))
        assert rel(got, Jo) <= (max(bound, 1e-12) if dtype == "f64" else 1e-3), (rel(got, Jo), bound)
