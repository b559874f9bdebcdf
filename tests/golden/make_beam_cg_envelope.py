"""Writes beam_cg_envelope.txt: the spread of the oracle's own iteration counts
for the paper's solver (outer CG, V(5,5), coarse CG with L-BFGS and the
spectral shift, ||F|| < 1e-6; Sec. 3) on the Neo-Hookean beam at the
refinement levels L1 and L2, when the initial state is perturbed at rounding
level.

At the twisted states of this problem the coarse CG meets negative curvature,
and the step at which it does depends on rounding; that step decides the
Rayleigh quotient, the shift and the coarse correction (Alg. 1), so the
preconditioner is a rounding-driven operator and the outer CG counts scatter.
Run 0 is the unperturbed boundary state; run s > 0 adds s-seeded N(0, 1) noise
of size 1e-13 to every entry that is not a Dirichlet value.  The GPU's counts
are compared with this envelope (tests/test_gpu_beam.py).

Only oracle/ is called.  Usage (from the repository root; 8 worker processes,
about two minutes):

    python -m tests.golden.make_beam_cg_envelope
"""
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RUNS = 17          # run 0 unperturbed, runs 1..16 perturbed
PERTURBATION = 1e-13
LEVELS = (1, 2)


def initial_state(k, seed):
    """The initial state of run `seed` at level L`k` (the GPU test starts from the
    same arrays)."""
    import numpy as np

    from oracle import hyper
    u0 = hyper.boundary_state(2 ** k)
    if seed > 0:
        fixed = hyper.dirichlet_mask(u0.shape)
        noise = np.random.default_rng(seed).standard_normal(u0.shape) * PERTURBATION
        u0 = np.where(fixed, u0, u0 + noise)
    return u0


def run(args):
    from oracle import jfnk
    k, seed = args
    _, st = jfnk.newton_solve(jfnk.build_hyper_hierarchy(k), initial_state(k, seed), jfnk.paper_options())
    assert st.converged, (k, seed)
    return k, seed, st.newton_its, st.linear_its, [int(c) for c in st.lin_hist]


def main():
    jobs = [(k, s) for k in LEVELS for s in range(RUNS)]
    with get_context("spawn").Pool(8) as pool:
        rows = pool.map(run, jobs)
    with open(os.path.join(HERE, "beam_cg_envelope.txt"), "w") as f:
        f.write("# Oracle iteration counts of the paper's solver on the Neo-Hookean beam (Sec. 3) at\n")
        f.write(f"# L1 and L2, initial state perturbed by {PERTURBATION:g} N(0,1) off the Dirichlet entries\n")
        f.write("# (run 0: unperturbed).  Written by tests/golden/make_beam_cg_envelope.py (oracle only).\n")
        f.write("# level  run  newton_its  cg_its  cg_per_newton_step\n")
        for k, s, ni, ci, hist in rows:
            f.write(f"L{k} {s} {ni} {ci} " + ",".join(str(c) for c in hist) + "\n")


def load():
    """{level k: [(run, newton_its, cg_its, [cg per Newton step]), ...]}"""
    out = {}
    with open(os.path.join(HERE, "beam_cg_envelope.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lv, s, ni, ci, hist = line.split()
            out.setdefault(int(lv[1:]), []).append((int(s), int(ni), int(ci), [int(c) for c in hist.split(",")]))
    return out


if __name__ == "__main__":
    main()
