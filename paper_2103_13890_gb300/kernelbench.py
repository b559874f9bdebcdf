"""Micro-benchmark of single hot-path operations through the C ABI.

    python -m paper_2103_13890_gb300.kernelbench --kind nd3d --n 160 --op smooth --dtype f64

op: residual | jvp | jvp_auto (the same with the FD step from the Sec. 1 formula:
    two masked reductions more, over u and v) | smooth (one Chebyshev application = start + fused steps)
    | vcycle | solve (a whole JFNK-MG solve from u0 = 0 to 1e-8, preconditioner
    in --dtype) | batch (the batched solve of 64 uneven 2D Bratu instances,
    sizes from {129^2, 257^2, 513^2} nodes, lambda ~ U[1, 6.5], seed 4)
    | sweep (residual and FD action over grid sizes, FP64 and FP32).
Prints one JSON line with the mean time per call (CUDA events
on the current stream, after warm-up) and, for the element kernels, the
achieved FP64/FP32 operation rate and HBM bandwidth of the algorithmic traffic.

--profiler-range brackets the timed calls with cudaProfilerStart/Stop, so that a
profiler started with profiling off captures exactly those launches.
"""
import argparse
import json

import torch

import paper_2103_13890_gb300 as jf

OPS_PER_ELEMENT = {"nd3d": 164, "ndk3d": 172, "bratu2d": 42}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="nd3d", choices=list(OPS_PER_ELEMENT))
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--levels", type=int, default=0, help="0: coarsest level with 4 elements")
    ap.add_argument("--op", default="residual",
                    choices=["residual", "jvp", "jvp_auto", "smooth", "vcycle", "solve", "batch", "sweep"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--profiler-range", action="store_true")
    ap.add_argument("--power-iters", type=int, default=30,
                    help="power-method iterations (at most, with --power-tol > 0)")
    ap.add_argument("--power-tol", type=float, default=1e-2,
                    help="stop the power method once successive estimates differ by less than this, "
                         "relative (Sec. 2: 30 and 1e-2); 0: always --power-iters")
    ap.add_argument("--batch-power-iters", type=int, default=10, help="--op batch: power-method iterations")
    ap.add_argument("--batch-power-tol", type=float, default=0.0, help="--op batch: stopping rule (0: off)")
    a = ap.parse_args()
    if a.op == "batch":
        return batch_main(a)
    if a.op == "sweep":
        return sweep_main(a)
    print(json.dumps(run_one(a)))


def run_one(a, restart=30):
    d = 2 if a.kind == "bratu2d" else 3
    n = a.n
    levels = a.levels
    if levels == 0:
        levels = 1
        while (n >> levels) >= 4 and ((n >> levels) << levels) == n:
            levels += 1
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    o = jf.default_options(pc_dtype=jf.F64 if a.dtype == "f64" else jf.F32,
                           eps_mode_pc=jf.EPS_PAPER if a.dtype == "f64" else jf.EPS_FP32,
                           nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=a.rtol, restart=restart,
                           power_iters=a.power_iters, power_tol=a.power_tol)
    kappa = None
    if a.kind == "ndk3d":
        g = torch.Generator().manual_seed(0)
        kappa = torch.exp(torch.randn((n,) * 3, generator=g, dtype=torch.float64))
    p = jf.Problem(a.kind, n, levels, lam=5.0, kappa=kappa, options=o)
    shape = (n + 1,) * d
    g = torch.Generator(device="cuda").manual_seed(1)
    u = (torch.rand(shape, generator=g, device="cuda", dtype=torch.float64) - 0.5) * 0.2
    bnd = torch.ones(shape, dtype=torch.bool, device="cuda")
    inner = tuple(slice(1, -1) for _ in range(d))
    bnd[inner] = False
    u[bnd] = 0.0
    v = torch.randn(shape, generator=g, device="cuda", dtype=torch.float64)
    v[bnd] = 0.0
    if a.op in ("smooth", "vcycle"):
        p.mg_setup(u, 0)
    uT, vT = u.to(dt), v.to(dt)
    F = p.residual(uT)
    out = torch.empty_like(uT)
    s = torch.zeros_like(uT)
    out64 = torch.empty_like(u)
    usol = torch.zeros_like(u)

    def call():
        if a.op == "residual":
            p.residual(uT, out=out)
        elif a.op == "jvp":
            p.jvp(uT, F, vT, out=out, eps=1e-7)
        elif a.op == "jvp_auto":
            p.jvp(uT, F, vT, out=out, eps_mode=jf.EPS_PAPER if a.dtype == "f64" else jf.EPS_FP32)
        elif a.op == "smooth":
            s.zero_()
            p.smooth(vT, s, level=levels - 1, nu=1, s_is_zero=True)
        elif a.op == "vcycle":
            p.mg_vcycle(v, out=out64)
        else:
            usol.zero_()
            return p.solve(usol)

    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.profiler_range:
        torch.cuda.profiler.start()
    e0.record()
    for _ in range(a.reps):
        st = call()
    e1.record()
    torch.cuda.synchronize()
    if a.profiler_range:
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / a.reps
    elems = n ** d
    w = 8 if a.dtype == "f64" else 4
    nodes = (n + 1) ** d
    stencils = {"residual": 1, "jvp": 1, "jvp_auto": 1, "smooth": o.cheb_degree - 1}.get(a.op)
    words = {"residual": 2 + (1 if a.kind == "nd3d" else 0), "jvp": 4, "jvp_auto": 6}.get(a.op)
    line = {"kind": a.kind, "n": n, "levels": levels, "op": a.op, "dtype": a.dtype, "ms": ms}
    if a.op == "solve":
        line.update(newton_its=st["newton_its"], fgmres_its=st["linear_its"], converged=st["converged"])
    if stencils:
        line["ops_per_s"] = OPS_PER_ELEMENT[a.kind] * elems * stencils / (ms * 1e-3)
    if words:
        line["gbs"] = words * w * nodes / (ms * 1e-3) / 1e9
    return line


def sweep_main(a):
    """Residual and FD-action throughput over grid sizes (where the roofline
    bends): 3D nonlinear diffusion on 65^3 .. 513^3 nodes and 2D Bratu on
    65^2 .. 4097^2 nodes, FP64 and FP32.  One JSON line per case with interior
    DOF/s, the fraction of the measured HBM bandwidth taken by the algorithmic
    bytes, and the fraction of the FP64 / FP32 pipe (152 SMs x 2 / 128
    operations per clock x 2070 MHz) taken by the element arithmetic."""
    import copy
    import os
    peaks = {}
    pf = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(pf):
        with open(pf) as f:
            peaks = json.load(f)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu = {"f64": 152 * 2 * 2.07e9, "f32": 152 * 128 * 2.07e9}
    cases = [("nd3d", n) for n in (64, 128, 256, 512)] + [("bratu2d", n) for n in (64, 256, 1024, 2048, 4096)]
    for kind, n in cases:
        for dt in ("f64", "f32"):
            for op in ("residual", "jvp"):
                b = copy.copy(a)
                b.kind, b.n, b.levels, b.op, b.dtype, b.reps = kind, n, 0, op, dt, max(3, min(a.reps, 20))
                line = run_one(b, restart=1)
                d = 2 if kind == "bratu2d" else 3
                line["dof_per_s"] = (n - 1) ** d / (line["ms"] * 1e-3)
                line["pct_hbm"] = 100.0 * line["gbs"] / hbm
                line["pct_alu"] = 100.0 * line["ops_per_s"] / alu[dt]
                print(json.dumps(line), flush=True)
                torch.cuda.empty_cache()


def batch_main(a):
    import math

    from workloads import batch_instances
    inst = batch_instances(64, seed=4)
    o = jf.default_options(rtol_newton=1e-8, pc_dtype=jf.F64 if a.dtype == "f64" else jf.F32,
                           eps_mode_pc=jf.EPS_PAPER if a.dtype == "f64" else jf.EPS_FP32,
                           power_iters=a.batch_power_iters, power_tol=a.batch_power_tol)
    ps = [jf.Problem("bratu2d", nn, int(round(math.log2(nn // 8))) + 1, lam=lam, options=o) for nn, lam in inst]
    us = [torch.zeros((nn + 1, nn + 1), dtype=torch.float64, device="cuda") for nn, _ in inst]

    def call():
        for x in us:
            x.zero_()
        return jf.solve_batched(ps, us, o)

    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.profiler_range:
        torch.cuda.profiler.start()
    e0.record()
    for _ in range(a.reps):
        st = call()
    e1.record()
    torch.cuda.synchronize()
    if a.profiler_range:
        torch.cuda.profiler.stop()
    print(json.dumps({"op": "batch", "instances": len(inst), "dtype": a.dtype, "ms": e0.elapsed_time(e1) / a.reps,
                      "converged": int(sum(s["converged"] for s in st))}))


if __name__ == "__main__":
    main()
