"""Host-side invariants of the halo-free 3D tiling (no GPU call): a small C++
program, compiled here with nvcc and linked against libjfnk.so, asks the
library for the tiling of every grid the halo-free kernels accept (n a multiple
of 32, 64..512) under every CTA cap and CTAs-per-SM setting, and checks that
the y tiles and z chunks cover the grid exactly, the face-buffer layout is the
one the kernels index, the paired FP32 kernel's CTA and shared memory fit, and
the block partials stay within the reduction scratch."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_halo_free_tiling_invariants(tmp_path):
    from paper_2103_13890_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    libdir = os.path.dirname(b.LIB)
    exe = str(tmp_path / "tiling_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-x", "cu", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2103_13890_gb300", "csrc"),
           os.path.join(ROOT, "tests", "host", "tiling_check.cu"), "-o", exe,
           "-L", libdir, "-ljfnk", "-Xlinker", "-rpath", "-Xlinker", libdir]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok 90"
