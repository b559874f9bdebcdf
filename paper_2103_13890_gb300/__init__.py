"""GB300 implementation of the Jacobian-free Newton-Krylov method with a
Jacobian-free geometric multigrid preconditioner (Kothari, Kopanicakova &
Krause, arXiv:2103.13890).

Every computation runs in libjfnk.so (hand-written CUDA for sm_103a, C ABI in
include/jfnk.h).  This module only marshals torch tensors (device memory and
the current CUDA stream) into those calls; it has no CPU fallback and raises
if the library is missing.

    import torch, paper_2103_13890_gb300 as jf
    p = jf.Problem("bratu2d", n_elem=64, levels=4, lam=5.0)
    u = torch.zeros(65, 65, dtype=torch.float64, device="cuda")
    stats = p.solve(u)            # u now holds the discrete solution

    # FP32 preconditioner inside the FP64 Newton/FGMRES loop
    o = jf.default_options(nu_pre=2, nu_post=2, cheb_degree=4, rtol_newton=1e-8,
                           pc_dtype=jf.F32, eps_mode_pc=jf.EPS_FP32)
    q = jf.Problem("nd3d", 128, 6, options=o)

    # the paper's own solver (outer CG, V(5,5), coarse CG with L-BFGS and the
    # spectral shift) on the hyperelastic beam
    b = jf.Problem("beam3d", 4, 3, options=jf.paper_options())

The single operations (residual, jvp, smooth, transfer, coarse_solve,
mg_setup, mg_vcycle, vjp) are methods of Problem; solve_batched solves many
2D instances together; autograd.JFNKSolve differentiates a solve with respect
to the coefficient field through the adjoint solve.
"""
import ctypes

import torch

from . import _abi
from ._abi import (BEAM3D, BRATU2D, COARSE_CGQN, COARSE_GMRES, EPS_FP32, EPS_PAPER, F32, F64,  # noqa: F401
                   KINDS, MINSURF2D, ND3D, NDK3D, OUTER_CG, OUTER_FGMRES)

_LIB = None


def lib():
    """The loaded libjfnk.so (ctypes), loaded on first use; raises if it is missing."""
    global _LIB
    if _LIB is None:
        _LIB = _abi.load_library()
    return _LIB


class JFNKError(RuntimeError):
    """A jfnk_status other than OK, with the library's thread-local message."""

    def __init__(self, status, msg):
        super().__init__(f"{_abi.STATUS.get(status, status)}: {msg}")
        self.status = status


def last_error():
    """The library's message for the last error on the calling thread."""
    return lib().jfnk_last_error().decode()


def _check(status):
    if status != 0:
        raise JFNKError(status, lib().jfnk_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def default_options(**kw):
    """jfnk_options with the library defaults, overridden by keyword."""
    o = _abi.Options()
    lib().jfnk_default_options(ctypes.byref(o))
    return _override(o, kw)


def paper_options(**kw):
    """jfnk_options with the paper's own settings (jfnk_paper_options: CG outer,
    V(5,5), [0.06, 1.2] lambda, coarse CG with L-BFGS and spectral shift,
    ||F|| < 1e-6), overridden by keyword."""
    o = _abi.Options()
    lib().jfnk_paper_options(ctypes.byref(o))
    return _override(o, kw)


def _override(o, kw):
    for k, v in kw.items():
        if k == "pc_dtype" and isinstance(v, torch.dtype):
            v = F32 if v == torch.float32 else F64
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _dtype_code(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def stats_dict(s):
    """jfnk_stats as a dict (histories cut to the iterations that ran)."""
    L = s.newton_its
    return {
        "newton_its": s.newton_its, "linear_its": s.linear_its, "status": _abi.STATUS.get(s.status, s.status),
        "converged": bool(s.converged), "res_hist": list(s.res_hist[:L + 1]),
        "alpha_hist": list(s.alpha_hist[:L]), "lin_hist": list(s.lin_hist[:L]), "ge": s.ge,
        "nF": list(s.nF), "nJv": list(s.nJv), "lambda_max": list(s.lambda_max), "solve_ms": s.solve_ms,
        "coarse_shifts": s.coarse_shifts, "coarse_negcurv": s.coarse_negcurv, "outer_negcurv": s.outer_negcurv,
        "ls_hist": list(s.ls_hist[:L]),
    }


class Problem:
    """One discretised problem on the current CUDA device with its workspace.

    kind: "bratu2d" | "nd3d" | "ndk3d" | "minsurf2d" | "beam3d"; n_elem: finest
    elements per direction (beam3d: across the beam, 10 n_elem along it, vectors of
    shape (n+1, n+1, 10n+1, 3));
    levels: multigrid levels; lam: Bratu lambda; load: optional FP64 finest
    load vector (nd3d); kappa: FP64 per-element coefficient (ndk3d, n_elem^3).
    options: the jfnk_options the workspace is laid out for (None: residual and
    jvp only)."""

    def __init__(self, kind, n_elem, levels, lam=0.0, load=None, kappa=None, options=None, device="cuda"):
        self.kind = kind
        self.d = 2 if kind in ("bratu2d", "minsurf2d") else 3
        self.n = n_elem
        self.levels = levels
        self.device = torch.device(device)
        self._keep = []
        desc = _abi.ProblemDesc()
        desc.kind = KINDS[kind]
        desc.n_elem = n_elem
        desc.levels = levels
        desc.lambda_ = lam
        if load is not None:
            load = load.to(self.device, torch.float64).contiguous()
            self._keep.append(load)
            desc.load = load.data_ptr()
        if kappa is not None:
            kappa = kappa.to(self.device, torch.float64).contiguous()
            self._keep.append(kappa)
            desc.kappa = kappa.data_ptr()
        self._h = ctypes.c_void_p()
        _check(lib().jfnk_problem_create(ctypes.byref(desc), ctypes.byref(self._h)))
        self.options = options
        opt_ref = ctypes.byref(options) if options is not None else None
        nbytes = ctypes.c_size_t()
        _check(lib().jfnk_workspace_size(self._h, opt_ref, ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        _check(lib().jfnk_set_workspace(self._h, opt_ref, _ptr(self.workspace), nbytes.value, _stream()))

    def shape(self, level=None):
        """Shape of a node vector of a level (finest by default): (n+1,)*d, or
        (m+1, m+1, 10m+1, 3) for the beam (axes z, y, x, component)."""
        lv = self.levels - 1 if level is None else level
        m = (self.n >> (self.levels - 1 - lv)) + 1
        if self.kind == "beam3d":
            return (m, m, 10 * (m - 1) + 1, 3)
        return (m,) * self.d

    def _lv(self, level):
        return self.levels - 1 if level is None else level

    def residual(self, u, level=None, out=None):
        """F(u) on a level (finest: A(u) - load; coarse: A(u))."""
        lv = self._lv(level)
        out = torch.empty_like(u) if out is None else out
        _check(lib().jfnk_residual(self._h, lv, _dtype_code(u), _ptr(u), _ptr(out), _stream()))
        return out

    def jvp(self, u, Fu, v, level=None, eps=0.0, eps_mode=EPS_PAPER, out=None):
        """(F(u + eps v) - F(u)) / eps with F(u) = Fu; eps <= 0 selects eps_mode."""
        lv = self._lv(level)
        out = torch.empty_like(u) if out is None else out
        _check(lib().jfnk_jvp(self._h, lv, _dtype_code(u), _ptr(u), _ptr(Fu), _ptr(v), _ptr(out),
                              float(eps), int(eps_mode), _stream()))
        return out

    def mg_setup(self, u, newton_step=0, options=None):
        """Set up the hierarchy at the finest-level iterate u (FP64): projected
        iterates x_l, A(x_l), the x statistics and the power-method estimates
        lambda_l (random start at newton_step 0, warm start after), Sec. 2."""
        o = options or self.options
        _check(lib().jfnk_mg_setup(self._h, ctypes.byref(o), _ptr(u), int(newton_step), _stream()))

    def mg_vcycle(self, b, out=None, options=None):
        """One V-cycle of Alg. 1 for J(u) s = b on the finest level (FP64 in and
        out); requires mg_setup."""
        o = options or self.options
        out = torch.empty_like(b) if out is None else out
        _check(lib().jfnk_mg_vcycle(self._h, ctypes.byref(o), _ptr(b), _ptr(out), _stream()))
        return out

    def transfer(self, op, x, level=None, out=None):
        """op: "restrict" | "project" (level -> level-1) or "prolong_add" (out(level) += I x)."""
        lv = self._lv(level)
        code = {"restrict": _abi.RESTRICT, "prolong_add": _abi.PROLONG_ADD, "project": _abi.PROJECT}[op]
        if out is None:
            if code == _abi.PROLONG_ADD:
                raise ValueError("prolong_add accumulates into out")
            out = torch.empty(self.shape(lv - 1), dtype=x.dtype, device=x.device)
        _check(lib().jfnk_transfer(self._h, code, lv, _dtype_code(x), _ptr(x), _ptr(out), _stream()))
        return out

    def smooth(self, b, s, level=None, nu=1, s_is_zero=False, options=None):
        """nu Chebyshev applications for J(x_l) s = b on a level, in place on s
        (vectors in the preconditioner dtype); requires mg_setup."""
        o = options or self.options
        _check(lib().jfnk_smooth(self._h, ctypes.byref(o), self._lv(level), _ptr(b), _ptr(s), int(nu),
                                 1 if s_is_zero else 0, _stream()))
        return s

    def coarse_solve(self, b, out=None, options=None):
        """The coarse-level solve of Alg. 1 (GMRES, or CG with L-BFGS and the
        spectral shift) for J(x_0) s = b; requires mg_setup."""
        o = options or self.options
        out = torch.empty_like(b) if out is None else out
        _check(lib().jfnk_coarse_solve(self._h, ctypes.byref(o), _ptr(b), _ptr(out), _stream()))
        return out

    def level_info(self, level):
        """lambda_max, sum |x_l| and ||x_l||_2 over the unknowns of a level."""
        lam, x1, x2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().jfnk_level_info(self._h, level, ctypes.byref(lam), ctypes.byref(x1), ctypes.byref(x2),
                                     _stream()))
        return {"lambda_max": lam.value, "sum_abs_x": x1.value, "norm2_x": x2.value}

    def level_vector(self, level, which):
        """which: "x" | "Ax" | "power" (preconditioner precision)."""
        dt = torch.float32 if self.options.pc_dtype == F32 else torch.float64
        out = torch.empty(self.shape(level), dtype=dt, device=self.device)
        code = {"x": 0, "Ax": 1, "power": 2}[which]
        _check(lib().jfnk_level_vector(self._h, level, code, _ptr(out), _stream()))
        return out

    def vjp(self, u, w, level=None, dkappa=False, out=None):
        """J(u)^T w (and (dF/dkappa)^T w per element when dkappa=True)."""
        lv = self._lv(level)
        out = torch.empty_like(u) if out is None else out
        dk = None
        if dkappa:
            m = self.n >> (self.levels - 1 - lv)
            dk = torch.empty((m,) * 3, dtype=u.dtype, device=u.device)
        _check(lib().jfnk_vjp(self._h, lv, _dtype_code(u), _ptr(u), _ptr(w), _ptr(out),
                              _ptr(dk) if dk is not None else None, _stream()))
        return (out, dk) if dkappa else out

    def set_kappa(self, kappa):
        """Replace the per-element coefficient of an NDK3D problem (copied to
        the workspace and averaged onto the coarse levels)."""
        kappa = kappa.to(self.device, torch.float64).contiguous()
        self._keep.append(kappa)
        self._keep = self._keep[-2:]
        _check(lib().jfnk_set_kappa(self._h, _ptr(kappa), _stream()))

    def adjoint_solve(self, u, g, rtol=1e-10, grad=True, options=None):
        """lambda with J(u)^T lambda = g, and grad_kappa = -(dF/dkappa)^T lambda."""
        o = options or self.options
        lam = torch.empty_like(u)
        gk = torch.empty((self.n,) * 3, dtype=torch.float64, device=u.device) if grad else None
        st = _abi.Stats()
        _check(lib().jfnk_adjoint_solve(self._h, ctypes.byref(o), _ptr(u), _ptr(g.contiguous()), _ptr(lam),
                                        _ptr(gk) if gk is not None else None, float(rtol), ctypes.byref(st),
                                        _stream()))
        return lam, gk, {"linear_its": st.linear_its, "ge": st.ge, "solve_ms": st.solve_ms}

    def solve(self, u, options=None, check=True):
        """Inexact JFNK solve in place on u (FP64, full node grid).  Returns stats."""
        o = options or self.options
        st = _abi.Stats()
        status = lib().jfnk_solve(self._h, ctypes.byref(o), _ptr(u), ctypes.byref(st), _stream())
        if check:
            _check(status)
        d = stats_dict(st)
        d["status_code"] = status
        return d

    def close(self):
        """Destroy the problem (host side; the workspace tensor is torch's)."""
        if self._h:
            lib().jfnk_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(problems, us, options=None, check=True):
    """Lock-step batched JFNK-MG solve of independent 2D Bratu problems
    (jfnk_solve_batched): one launch per level operation over all instances.
    us[i] (FP64 full node grid of problem i) is updated in place.  Returns the
    list of per-instance stats."""
    n = len(problems)
    o = options or problems[0].options
    hs = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
    ups = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
    st = (_abi.Stats * n)()
    status = lib().jfnk_solve_batched(hs, n, ctypes.byref(o), ups, st, _stream())
    if check:
        _check(status)
    return [stats_dict(s) for s in st]


def jvp_noalloc(kind, u, Fu, v, lam=0.0, kappa=None, load=None, eps=0.0, eps_mode=EPS_PAPER, out=None):
    """FD Jacobian action without a problem object or workspace (jfnk_jvp_noalloc),
    for callers that cannot allocate device memory; kappa and load must have u's
    dtype.  Calls that overlap on the GPU share the library's fixed scratch."""
    n = u.shape[0] - 1
    out = torch.empty_like(u) if out is None else out
    kp = _ptr(kappa) if kappa is not None else None
    lp = _ptr(load) if load is not None else None
    _check(lib().jfnk_jvp_noalloc(KINDS[kind], n, float(lam), kp, lp, _dtype_code(u), _ptr(u), _ptr(Fu), _ptr(v),
                                  _ptr(out), float(eps), int(eps_mode), _stream()))
    return out


def measure_peaks():
    """Measured FMA/s of the current GPU: {"fp64", "fp32", "fp32x2"} (FMA chains
    on every SM, jfnk_measure_peaks)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().jfnk_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream()))
    return {"fp64": a.value, "fp32": b.value, "fp32x2": c.value}


def debug_bounds(reset=True):
    """(enabled, first out-of-range source line or 0, message) of a bounds-checked
    build (jfnk_debug_bounds); enabled is False in a normal build."""
    en, line = ctypes.c_int(), ctypes.c_uint()
    _check(lib().jfnk_debug_bounds(ctypes.byref(en), ctypes.byref(line), 1 if reset else 0))
    return bool(en.value), line.value, last_error() if line.value else ""


def kernel_launches(reset=False):
    """Kernels the library has launched (graph replays count their kernels);
    reset=True returns the count and restarts it."""
    return lib().jfnk_kernel_launches(1 if reset else 0)


def profile_enable(on=True):
    """Bracket every element-kernel launch with CUDA events on its stream (see
    profile_read); V-cycles then launch directly instead of from their graph."""
    lib().jfnk_profile_enable(1 if on else 0)


def profile_read(max_classes=256):
    """{class name: (launches, total_ms, elements_per_launch)} of the event profile."""
    nl = 96
    names = ctypes.create_string_buffer(max_classes * nl)
    cnt = (ctypes.c_longlong * max_classes)()
    ms = (ctypes.c_double * max_classes)()
    work = (ctypes.c_double * max_classes)()
    n = lib().jfnk_profile_read(max_classes, names, nl, cnt, ms, work)
    out = {}
    for i in range(min(n, max_classes)):
        name = names.raw[i * nl:(i + 1) * nl].split(b"\0", 1)[0].decode()
        out[name] = (cnt[i], ms[i], work[i])
    return out
