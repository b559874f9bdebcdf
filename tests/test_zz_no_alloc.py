"""jfnk_jvp_noalloc, the FD Jacobian action for callers that cannot allocate
device memory (no problem object, no workspace; its scratch is a fixed array
inside libjfnk.so), gives the same result as jfnk_jvp, call after call.

This file is collected last so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process (the first
call on the device looks the scratch up) and after the other tests."""
import numpy as np
import pytest

from gpu_common import dev, host, jf, kernel_path, rel, torch
from oracle import fem
from workloads import random_direction, random_state_field

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,dtype", [("nd3d", 33, "f64"), ("ndk3d", 20, "f64"), ("bratu2d", 95, "f32"),
                                          ("nd3d", 40, "f32")])
def test_jvp_noalloc_matches_jvp_on_two_calls_in_a_row(kind, n, dtype, monkeypatch):
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
    for call in range(2):
        v = random_direction(n, d, seed=100 + call)
        vd = dev(v, tdt)
        ref = host(p.jvp(ud, Fu, vd))
        got = host(jf().jvp_noalloc(kind, ud, Fu, vd, lam=5.0, kappa=kd, load=ld))
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
