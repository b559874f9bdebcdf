"""The C ABI library builds, loads and exports every symbol include/jfnk.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "jfnk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jfnk_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_13890_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jfnk_\w+)", out))
    assert set(names) <= exported


def test_python_binding_covers_header(libpath):
    from paper_2103_13890_gb300 import _abi
    bound = {s[0] for s in _abi.SIGNATURES}
    assert set(_declared()) <= bound


def test_host_side_errors_without_gpu(libpath):
    """Argument validation happens on the host and reports a status + message."""
    from paper_2103_13890_gb300 import _abi
    lib = _abi.load_library(libpath)
    desc = _abi.ProblemDesc(kind=7, n_elem=8, levels=2)
    h = ctypes.c_void_p()
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    assert b"kind" in lib.jfnk_last_error()
    desc = _abi.ProblemDesc(kind=0, n_elem=12, levels=4)  # 12 / 8 not integral
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    desc = _abi.ProblemDesc(kind=2, n_elem=8, levels=2)  # NDK without kappa
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    desc = _abi.ProblemDesc(kind=0, n_elem=64, levels=4)
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 0
    o = _abi.Options()
    lib.jfnk_default_options(ctypes.byref(o))
    assert o.nu_pre == 3 and o.cheb_degree == 3 and o.restart == 30 and abs(o.cheb_lo - 0.1) < 1e-15
    nb = ctypes.c_size_t()
    assert lib.jfnk_workspace_size(h, ctypes.byref(o), ctypes.byref(nb)) == 0 and nb.value > 0
    nb0 = ctypes.c_size_t()
    assert lib.jfnk_workspace_size(h, None, ctypes.byref(nb0)) == 0 and nb0.value < nb.value
    o.restart = 0
    assert lib.jfnk_workspace_size(h, ctypes.byref(o), ctypes.byref(nb)) == 1
    # no workspace attached: calls fail cleanly
    assert lib.jfnk_residual(h, 3, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == 9
    assert lib.jfnk_problem_destroy(h) == 0


def test_paper_options_and_their_validation(libpath):
    """The paper's own settings (Sec. 2, Sec. 3 "Setup") as the library states
    them, and the host-side checks of the options that select them."""
    from paper_2103_13890_gb300 import _abi
    lib = _abi.load_library(libpath)
    o = _abi.Options()
    lib.jfnk_paper_options(ctypes.byref(o))
    assert (o.nu_pre, o.nu_post, o.cheb_degree) == (1, 1, 5)  # one degree-5 polynomial a side
    assert (o.cheb_lo, o.cheb_hi) == (0.06, 1.2)
    assert (o.power_iters, o.power_tol) == (30, 1e-2)
    assert (o.rtol_newton, o.atol_newton) == (0.0, 1e-6)
    assert (o.outer, o.coarse_method, o.lbfgs_pairs, o.shift_gamma) == (
        _abi.OUTER_CG, _abi.COARSE_CGQN, 20, 5.0)
    desc = _abi.ProblemDesc(kind=_abi.BRATU2D, n_elem=100, levels=3)
    h = ctypes.c_void_p()
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 0
    nb = ctypes.c_size_t()
    assert lib.jfnk_workspace_size(h, ctypes.byref(o), ctypes.byref(nb)) == 0 and nb.value > 0
    for field, bad in (("outer", 7), ("coarse_method", 9), ("lbfgs_pairs", 0), ("lbfgs_pairs", 10 ** 6),
                       ("shift_gamma", 1.0), ("cheb_lo", 0.0), ("cheb_hi", 0.05)):
        q = _abi.Options()
        lib.jfnk_paper_options(ctypes.byref(q))
        setattr(q, field, bad)
        assert lib.jfnk_workspace_size(h, ctypes.byref(q), ctypes.byref(nb)) == 1, field
        assert b"invalid options" in lib.jfnk_last_error()
    assert lib.jfnk_problem_destroy(h) == 0


def test_beam_and_minimal_surface_problems_on_the_host(libpath):
    """The Sec. 3 problems the paper adds: the beam's 10m x m x m grid (3 values
    a node) and the minimal surface are created and sized without a GPU."""
    from paper_2103_13890_gb300 import _abi
    lib = _abi.load_library(libpath)
    h = ctypes.c_void_p()
    nb = ctypes.c_size_t()
    for kind, n, levels in ((_abi.BEAM3D, 4, 3), (_abi.BEAM3D, 1, 1), (_abi.MINSURF2D, 100, 3)):
        desc = _abi.ProblemDesc(kind=kind, n_elem=n, levels=levels)
        assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 0, lib.jfnk_last_error()
        assert lib.jfnk_workspace_size(h, None, ctypes.byref(nb)) == 0 and nb.value > 0
        assert lib.jfnk_problem_destroy(h) == 0
    # three beam levels need 2^2 | n: n = 2 leaves a coarse grid of less than one element
    desc = _abi.ProblemDesc(kind=_abi.BEAM3D, n_elem=2, levels=3)
    assert lib.jfnk_problem_create(ctypes.byref(desc), ctypes.byref(h)) == 1
