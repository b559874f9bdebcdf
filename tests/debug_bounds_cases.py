"""Odd-size cases of every kernel path, run against the bounds-checked build of
the library (JFNK_LIB must point to it).  Prints one JSON line with the bounds
record (jfnk_debug_bounds) after all cases.  Run by test_gpu_debug_bounds.py in
a child process, so that the normal build stays loaded in the test session."""
import json
import os
import sys

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2103_13890_gb300 as jf  # noqa: E402

PATHS = {
    "default": {},
    "ep": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "0"},
    "zm": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "2",
           "JFNK_ZM3D_MIN_N_F32": "2"},
    "tiled": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0"},
    "v2": {"JFNK_EP3D_MAX_N_F64": "0", "JFNK_EP3D_MAX_N_F32": "0", "JFNK_V3_F32": "0"},
    "cluster": {"JFNK_EP3D_MAX_N_F64": "100000", "JFNK_EP3D_MAX_N_F32": "100000", "JFNK_ZM3D_MIN_N_F64": "0",
                "JFNK_EP3D_CLUSTER_MIN_N": "2", "JFNK_EP3D_CLUSTER_MAX_N": "32"},
}


def set_path(name):
    for k in ("JFNK_EP3D_MAX_N_F64", "JFNK_EP3D_MAX_N_F32", "JFNK_ZM3D_MIN_N_F64", "JFNK_ZM3D_MIN_N_F32",
              "JFNK_V3_F32", "JFNK_EP3D_CLUSTER_MIN_N", "JFNK_EP3D_CLUSTER_MAX_N"):
        os.environ.pop(k, None)
    os.environ.update(PATHS[name])


def levels_for(n, coarse):
    lv = 1
    while (n >> lv) >= coarse and ((n >> lv) << lv) == n:
        lv += 1
    return lv


def field(shape, dtype, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return (torch.rand(shape, generator=g, device="cuda", dtype=torch.float64) - 0.5).to(dtype)


def main():
    cases = 0
    for path in PATHS:
        set_path(path)
        for kind, n in (("bratu2d", 7), ("bratu2d", 95), ("bratu2d", 96), ("nd3d", 4), ("nd3d", 33), ("nd3d", 37),
                        ("ndk3d", 5), ("ndk3d", 37), ("nd3d", 64), ("nd3d", 96)):
            d = 2 if kind == "bratu2d" else 3
            kap = torch.rand((n,) * 3, dtype=torch.float64) + 0.5 if kind == "ndk3d" else None
            p = jf.Problem(kind, n, 1, lam=5.0, kappa=kap)
            for dt in (torch.float64, torch.float32):
                u = field((n + 1,) * d, dt, 1)
                v = field((n + 1,) * d, dt, 2)
                F = p.residual(u)
                p.jvp(u, F, v)
                cases += 2
        # multigrid building blocks and solves on hierarchies with odd coarse sizes
        for kind, n, coarse in (("bratu2d", 48, 3), ("nd3d", 24, 3), ("nd3d", 96, 3)):
            d = 2 if kind == "bratu2d" else 3
            for pc in (jf.F64, jf.F32):
                o = jf.default_options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=1e-8, pc_dtype=pc,
                                       eps_mode_pc=jf.EPS_PAPER if pc == jf.F64 else jf.EPS_FP32)
                p = jf.Problem(kind, n, levels_for(n, coarse), lam=5.0, options=o)
                u = torch.zeros((n + 1,) * d, dtype=torch.float64, device="cuda")
                st = p.solve(u)
                assert st["converged"], st
                cases += 1
    # the batched solver and the beam
    set_path("default")
    o = jf.default_options(rtol_newton=1e-8, pc_dtype=jf.F32, eps_mode_pc=jf.EPS_FP32)
    ps = [jf.Problem("bratu2d", n, levels_for(n, 8), lam=lam, options=o) for n, lam in ((32, 5.0), (64, 2.0))]
    us = [torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda") for n in (32, 64)]
    jf.solve_batched(ps, us, o)
    cases += 1
    b = jf.Problem("beam3d", 2, 2, options=jf.paper_options())
    ub = torch.zeros(b.shape(), dtype=torch.float64, device="cuda")
    b.residual(ub)
    cases += 1
    torch.cuda.synchronize()
    enabled, line, msg = jf.debug_bounds()
    print(json.dumps({"enabled": enabled, "line": line, "message": msg, "cases": cases}))


if __name__ == "__main__":
    main()
