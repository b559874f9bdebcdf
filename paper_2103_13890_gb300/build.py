"""Build libjfnk.so in-tree for sm_103a (GB300).

Each CUDA translation unit under csrc/ is compiled by its own nvcc process in
parallel, then linked into paper_2103_13890_gb300/lib/libjfnk.so.  No cmake.

    python -m paper_2103_13890_gb300.build [--verbose-ptxas] [--debug-bounds]

--debug-bounds builds the bounds-checked variant (-DJFNK_DEBUG_BOUNDS: every
checked index out of range is recorded and clamped, see jfnk_debug_bounds) into
lib/debug/libjfnk.so; the package loads it when JFNK_LIB points there.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libjfnk.so")
DEBUG_DIR = os.path.join(LIBDIR, "debug")
DEBUG_LIB = os.path.join(DEBUG_DIR, "libjfnk.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src, ptxas_verbose, objdir, extra):
    obj = os.path.join(objdir, src[:-3] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if ptxas_verbose else []) + \
        ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def build(ptxas_verbose=False, quiet=True, debug_bounds=False):
    """Compile every translation unit and link libjfnk.so (the bounds-checked
    variant with debug_bounds); returns the library path."""
    objdir = os.path.join(DEBUG_DIR, "obj") if debug_bounds else OBJDIR
    lib = DEBUG_LIB if debug_bounds else LIB
    extra = ["-DJFNK_DEBUG_BOUNDS"] if debug_bounds else []
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda s: _compile(s, ptxas_verbose, objdir, extra), srcs))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, out in results:
        if (rc != 0 or not quiet) and out.strip():
            sys.stderr.write(f"--- {src}\n{out}\n")
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(r[0] for r in failed))
    objs = [r[1] for r in results]
    link = [nvcc()] + ARCH + ["-shared", "-o", lib] + objs
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libjfnk.so failed")
    return lib


if __name__ == "__main__":
    print(build(ptxas_verbose="--verbose-ptxas" in sys.argv, quiet="--verbose-ptxas" not in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
