"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def jf():
    import paper_2103_13890_gb300 as m
    return m


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# 3D kernel selection (read when a Problem is created): "ep" runs the
# element-parallel kernels (one element a thread) on every 3D level, "zm" their
# z-marching variant (element columns) wherever the element-parallel kernels
# run (n > 8 in FP32), "tiled" the halo-free kernel (n a multiple of 32,
# n >= 64; in FP32 its two-elements-per-thread variant) or the tiled one, "v2"
# the same with the one-element-per-thread halo-free kernel in FP32 too,
# "default" the library's choice.
KERNEL_PATHS = {
    "default": {},
    "ep": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "0",
           "JFNK_ZM3D_MIN_N_F32": "0", "JFNK_EP3D_CLUSTER_MAX_N": "0"},
    "zm": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "2",
           "JFNK_ZM3D_MIN_N_F32": "2", "JFNK_EP3D_CLUSTER_MAX_N": "0"},
    # FP32 element-parallel levels with n <= 32 in one thread-block cluster
    # (the FP64 levels as on "ep")
    "cluster": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "0",
                "JFNK_ZM3D_MIN_N_F32": "0", "JFNK_EP3D_CLUSTER_MIN_N": "2", "JFNK_EP3D_CLUSTER_MAX_N": "32"},
    "tiled": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0"},
    "v2": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0", "JFNK_V3_F32": "0"},
    # the two-elements-per-thread kernel with one / two CTAs per SM in every
    # mode (by default the residual takes two and the other modes one)
    "v3one": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0", "JFNK_V3_F32": "1"},
    "v3two": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0", "JFNK_V3_F32": "2"},
    # the per-mode choice of the default
    "v3mixed": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0", "JFNK_V3_F32": "3"},
}


def kernel_path(monkeypatch, path):
    for k in ("JFNK_EP3D_MAX_N_F64", "JFNK_EP3D_MAX_N_F32", "JFNK_V3_F32", "JFNK_ZM3D_MIN_N_F64",
              "JFNK_ZM3D_MIN_N_F32", "JFNK_EP3D_CLUSTER_MIN_N", "JFNK_EP3D_CLUSTER_MAX_N"):
        monkeypatch.delenv(k, raising=False)
    for k, v in KERNEL_PATHS[path].items():
        monkeypatch.setenv(k, v)
