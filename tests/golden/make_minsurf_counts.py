"""Writes minsurf_counts.txt: the oracle's Newton and CG iteration counts and GE
of the paper's own solver (outer CG, V(5,5), coarse CG with L-BFGS and the
spectral shift, ||F|| < 1e-6; Sec. 3) on the minimal-surface problem at the
refinement levels L1..L5 (25 * 2^k elements per direction, k + 1 levels).

Only oracle/ is called.  Usage (from the repository root, about 7 minutes):

    python -m tests.golden.make_minsurf_counts
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import fem, jfnk  # noqa: E402


def main():
    rows = []
    for k in range(1, 6):
        n = 25 * 2 ** k
        t0 = time.perf_counter()
        lv = jfnk.build_hierarchy("minsurf2d", n, k + 1)
        _, st = jfnk.newton_solve(lv, fem.minsurf_boundary(n), jfnk.paper_options())
        assert st.converged, (k, st)
        rows.append((k, n, st.newton_its, st.linear_its, st.ge, time.perf_counter() - t0))
    with open(os.path.join(HERE, "minsurf_counts.txt"), "w") as f:
        f.write("# Oracle counts of the paper's solver on the minimal surface (Sec. 3), written by\n")
        f.write("# tests/golden/make_minsurf_counts.py (oracle only).\n")
        f.write("# level  n_elem  newton_its  cg_its  ge  seconds\n")
        for k, n, ni, ci, ge, dt in rows:
            f.write(f"L{k} {n} {ni} {ci} {ge:.3f} {dt:.1f}\n")


def load():
    """{level k: (newton_its, cg_its, ge)}"""
    out = {}
    with open(os.path.join(HERE, "minsurf_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            out[int(t[0][1:])] = (int(t[2]), int(t[3]), float(t[4]))
    return out


if __name__ == "__main__":
    main()
