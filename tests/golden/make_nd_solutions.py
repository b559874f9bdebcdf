"""Writes nd3d_solution_<n+1>.txt: sampled nodal values of the oracle's
converged discrete solution of the 3D nonlinear-diffusion workload.

Problem: -div((1+u^2) grad u) = f on the unit cube, f manufactured from
u* = sin(pi x) sin(pi y) sin(pi z), homogeneous Dirichlet data, Q1 elements,
2x2x2 Gauss points (oracle.fem).  Solver: the oracle's JFNK with the
Jacobian-free V(2,2)-cycle of Alg. 1 (Chebyshev degree 4, FP64 throughout),
FGMRES(30), from u0 = 0, driven to a 1e-12 relative nonlinear residual, so the
stored values are the discrete solution to ~1e-13 (quadratic convergence).

Only oracle/ is called.  Usage (from the repository root):

    python -m tests.golden.make_nd_solutions 64 5     # 65^3 nodes, 5 levels (~1.5 min)
    python -m tests.golden.make_nd_solutions 128 6    # 129^3 nodes, 6 levels (~15 min)

File format: '#' comment lines (settings, counts, norms of the full solution),
then one line per sampled interior node: flat index (x fastest) and value.
The sampled nodes are every fourth of 4096 interior nodes drawn without
replacement by numpy's PCG64 with seed 20210325 and sorted (1024 nodes).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import fem, jfnk  # noqa: E402

SAMPLES = 4096
SEED = 20210325


def sample_indices(n):
    """Flat indices of the sampled interior nodes of the (n+1)^3 grid."""
    interior = np.flatnonzero(fem.interior(((n + 1),) * 3).ravel())
    rng = np.random.Generator(np.random.PCG64(SEED))
    return np.sort(rng.choice(interior, size=min(SAMPLES, interior.size), replace=False))[::4]


def main(n, levels):
    t0 = time.perf_counter()
    lv = jfnk.build_hierarchy("nd3d", n, levels, load=fem.mms_load(n))
    o = jfnk.Options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=1e-12, max_newton=30)
    u, st = jfnk.newton_solve(lv, np.zeros((n + 1,) * 3), o)
    dt = time.perf_counter() - t0
    assert st.converged, st
    idx = sample_indices(n)
    path = os.path.join(HERE, f"nd3d_solution_{n + 1}.txt")
    with open(path, "w") as f:
        f.write("# Oracle solution of the 3D nonlinear-diffusion workload (manufactured u*),\n")
        f.write(f"# {n + 1}^3 nodes, {levels} levels, V(2,2) Chebyshev degree 4, FGMRES(30),\n")
        f.write("# rtol 1e-12; written by tests/golden/make_nd_solutions.py (oracle only).\n")
        f.write(f"# newton_its {st.newton_its}  fgmres_its {st.linear_its}  ge {st.ge:.3f}  "
                f"final_rel_residual {st.res_hist[-1] / st.res_hist[0]:.3e}  seconds {dt:.1f}\n")
        f.write(f"# norm2 {np.linalg.norm(u):.17e}\n")
        f.write(f"# normmax {np.abs(u).max():.17e}\n")
        f.write(f"# sum {u.sum():.17e}\n")
        f.write(f"# samples {idx.size} seed {SEED}\n")
        flat = u.ravel()
        for i in idx:
            f.write(f"{int(i)} {flat[i]:.17e}\n")
    print(path, st.newton_its, st.linear_its, f"{dt:.1f}s")


def load(n_nodes):
    """(indices, values, header dict) of nd3d_solution_<n_nodes>.txt."""
    hdr, idx, val = {}, [], []
    with open(os.path.join(HERE, f"nd3d_solution_{n_nodes}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                t = line[1:].split()
                if len(t) == 2 and t[0] in ("norm2", "normmax", "sum"):
                    hdr[t[0]] = float(t[1])
                continue
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    return np.array(idx, dtype=np.int64), np.array(val), hdr


if __name__ == "__main__":
    main(int(sys.argv[1]), int(sys.argv[2]))
