"""The bounds-checked build (-DJFNK_DEBUG_BOUNDS) runs odd-size cases of every
kernel path (residual and FD action in both precisions, the element-parallel,
z-marching, halo-free and tiled 3D kernels, the 2D kernel, transfers, solves
with odd coarse grids, the batched solver) without recording an index out of
range.  The checks clamp and record instead of faulting, so the run is safe
even if an index were wrong.  The variant is built on first use (about a
minute) and loaded in a child process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_no_index_out_of_range_in_the_bounds_checked_build():
    sys.path.insert(0, ROOT)
    from paper_2103_13890_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, JFNK_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    assert rec["enabled"], rec
    assert rec["cases"] > 100
    assert rec["line"] == 0, rec
