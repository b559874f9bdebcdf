"""Jacobian-free Newton-Krylov with a Jacobian-free multigrid preconditioner (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Plain FP64 restatement, in the paper's order and notation:
  Sec. 1     Newton x^(k+1) = x^(k) + alpha dx^(k); J dx = -F; FD Jacobian action
             J(x)u ~ (F(x + eps u) - F(x)) / eps with
             eps = (1/(n ||u||_2)) sum_i sqrt(eps_p) (1 + |x_i|).
  Sec. 2     transfer operators (oracle.transfer), Chebyshev smoother on
             [c_lo lambda_l, c_hi lambda_l], power method for lambda_l
             (random start at the first Newton step, warm start afterwards),
             Krylov coarse solve.
  Alg. 1     the V(nu1, nu2)-cycle MG(x_l, F(x_l), b_l, l).
  Sec. 3     inexact Newton with cubic backtracking, forcing
             ||J dx + F|| <= eta ||F||, gradient-evaluation count
             GE = sum_l 2^(-d(L-l)) GE_l.

Readings (the paper is silent or differs from the configured workloads):
  * n in the eps formula counts interior unknowns; sums run over interior nodes.
  * "fp32" eps mode: eps = sqrt(2^-23) (1 + ||x||_2) / ||u||_2 (used by the
    single-precision preconditioner; evaluated here in FP64).
  * ||u|| = 0 gives J u = 0.
  * Chebyshev: the classical three-term recurrence (Saad, Iterative Methods for
    Sparse Linear Systems, 2nd ed., Sec. 12.3) with no diagonal scaling;
    "nu smoothing steps with degree k" = nu applications of the degree-k
    polynomial, each restarted from the current iterate.
  * Power method: lambda = ||J v|| for ||v|| = 1 after a fixed number of
    iterations, or the paper's stopping rule |lambda_i - lambda_(i-1)| < tol
    read relative to lambda_i.
  * Coarse solve: unrestarted GMRES (the configured workloads use GMRES where
    the paper uses CG), x0 = 0, modified Gram-Schmidt, stop at
    ||r|| <= tol ||r_0|| (relative reading) or after n_0 iterations.
  * Outer Krylov: right-preconditioned flexible GMRES(m) (the configured
    workloads; the paper uses CG because its J is symmetric).
  * Forcing term: eta = min(0.5, ||F_k|| / ||F_0||) (relative reading of
    eta = min(0.5, ||F||)); the paper's absolute form is an option.
  * Line search: backtracking with quadratic then cubic interpolation
    (Dennis & Schnabel, Numerical Methods for Unconstrained Optimization and
    Nonlinear Equations, Sec. 6.3) on phi(alpha) = 1/2 ||F(u + alpha dx)||^2,
    slope phi'(0) = F . (J dx) from one FD action, Armijo constant 1e-4,
    new step clipped to [0.1, 0.5] alpha, at most 10 backtracks.
  * P x^(k) and F(P x^(k)) on each level are evaluated once per Newton step
    (x^(k) does not change during the step, so this equals re-evaluating
    them inside every cycle as Alg. 1 writes it).
"""
from dataclasses import dataclass, field

import numpy as np

from . import fem, transfer
from .splitmix import start_vector

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


@dataclass
class Options:
    nu_pre: int = 3
    nu_post: int = 3
    cheb_degree: int = 3
    cheb_lo: float = 0.1
    cheb_hi: float = 1.1
    power_iters: int = 10
    power_tol: float = 0.0          # > 0: paper rule (stop when relative change < tol)
    restart: int = 30
    max_linear: int = 300           # total FGMRES iterations per Newton step
    rtol_newton: float = 1e-8
    atol_newton: float = 0.0        # > 0: paper's absolute stop ||F|| < atol
    eta_mode: str = "relative"      # or "paper"
    eta_max: float = 0.5
    coarse_tol: float = 1e-12
    coarse_tol_mode: str = "relative"  # or "absolute"
    coarse_maxit: int = 0           # 0: number of coarse unknowns
    eps_mode_pc: str = "paper"      # "paper" or "fp32": eps used inside the preconditioner
    max_newton: int = 50
    line_search: bool = True
    ls_max: int = 10
    seed: int = 0


# ---------------------------------------------------------------------------
# Level hierarchy {T_l}, l = 0 (coarsest) .. L (finest)   (Sec. 2)
# ---------------------------------------------------------------------------

class Level:
    def __init__(self, kind, n, lam, kappa, load):
        self.kind = kind
        self.n = n
        self.d = fem.dim_of(kind)
        self.lam = lam
        self.kappa = kappa
        self.load = load
        self.shape = (n + 1,) * self.d
        self.mask = fem.interior(self.shape)
        self.n_unknowns = (n - 1) ** self.d
        self.ge = 0          # gradient evaluations on this level
        self.x = None
        self.Fx = None
        self.lam_max = None
        self.power_v = None

    def F(self, x):
        self.ge += 1
        return fem.residual(self.kind, x, self.lam, self.kappa, self.load)


def build_hierarchy(kind, n_finest, n_levels, lam=0.0, kappa=None, load=None):
    """Levels l = 0..L with n_l = n_finest / 2^(L-l) elements per direction.
    Coarse levels rediscretise the same PDE (Sec. 2, geometric MG): nd3d uses
    the manufactured load of that level, ndk3d the arithmetic-mean coefficient."""
    L = n_levels - 1
    levels = [None] * n_levels
    kap = kappa
    for l in range(L, -1, -1):
        n = n_finest >> (L - l)
        assert n << (L - l) == n_finest and n >= 2
        if kind == "nd3d":
            ld = load if (l == L and load is not None) else fem.mms_load(n)
        else:
            ld = None
        levels[l] = Level(kind, n, lam, kap, ld)
        if kap is not None and l > 0:
            kap = transfer.coarsen_kappa(kap)
    return levels


def total_ge(levels):
    """GE = sum_l 2^(-d(L-l)) GE_l  (Sec. 3)."""
    L = len(levels) - 1
    d = levels[0].d
    return sum(2.0 ** (-d * (L - l)) * lv.ge for l, lv in enumerate(levels))


# ---------------------------------------------------------------------------
# FD Jacobian action (Sec. 1)
# ---------------------------------------------------------------------------

def norm_i(v, mask):
    return float(np.sqrt(np.sum(v[mask] ** 2)))


def fd_eps(x, v, mask, mode="paper"):
    """The finite-difference step.
    paper: eps = (1/(n ||v||_2)) sum_i sqrt(eps_p)(1 + |x_i|), eps_p = 2^-52, n interior unknowns.
    fp32:  eps = sqrt(2^-23) (1 + ||x||_2) / ||v||_2."""
    nv = norm_i(v, mask)
    if nv == 0.0:
        return 0.0
    if mode == "paper":
        n = int(mask.sum())
        return float(np.sum(np.sqrt(EPS64) * (1.0 + np.abs(x[mask])))) / (n * nv)
    if mode == "fp32":
        return np.sqrt(EPS32) * (1.0 + norm_i(x, mask)) / nv
    raise ValueError(mode)


def fd_jv(level, x, Fx, v, mode="paper", eps=None):
    """J(x) v ~ (F(x + eps v) - F(x)) / eps, v restricted to interior nodes."""
    v = np.where(level.mask, v, 0.0)
    if eps is None:
        eps = fd_eps(x, v, level.mask, mode)
    if eps == 0.0:
        return np.zeros_like(v)
    return (level.F(x + eps * v) - Fx) / eps


# ---------------------------------------------------------------------------
# Power method for lambda_l (Sec. 2, "Smoothers")
# ---------------------------------------------------------------------------

def power_method(level, x, Fx, v0, iters, mode="paper", tol=0.0):
    """Estimate the largest eigenvalue of J(x) on this level.  v is normalised,
    w = J v, lambda = ||w||, v <- w / ||w||.  Returns (lambda, v)."""
    v = np.where(level.mask, v0, 0.0)
    v = v / norm_i(v, level.mask)
    lam = 0.0
    for _ in range(iters):
        w = fd_jv(level, x, Fx, v, mode)
        lam_new = norm_i(w, level.mask)
        if lam_new == 0.0:
            return 0.0, v
        v = w / lam_new
        done = tol > 0.0 and lam > 0.0 and abs(lam_new - lam) < tol * lam_new
        lam = lam_new
        if done:
            break
    return lam, v


# ---------------------------------------------------------------------------
# Chebyshev smoother (Sec. 2, "Smoothers")
# ---------------------------------------------------------------------------

def chebyshev(level, s, x, Fx, b, nu, degree, lam_max, lo, hi, mode="paper"):
    """nu applications of the degree-k Chebyshev polynomial iteration for
    J(x) s = b on [lo*lam_max, hi*lam_max], each restarted from the current s
    (three-term recurrence of Saad, Sec. 12.3)."""
    a_ = lo * lam_max
    b_ = hi * lam_max
    theta = 0.5 * (b_ + a_)
    delta = 0.5 * (b_ - a_)
    sigma = theta / delta
    for _ in range(nu):
        if np.any(s[level.mask] != 0.0):
            r = b - fd_jv(level, x, Fx, s, mode)
        else:
            r = b.copy()
        r = np.where(level.mask, r, 0.0)
        rho = 1.0 / sigma
        d = r / theta
        for i in range(degree):
            s = s + d
            if i < degree - 1:
                r = r - fd_jv(level, x, Fx, d, mode)
                rho_new = 1.0 / (2.0 * sigma - rho)
                d = rho_new * rho * d + (2.0 * rho_new / delta) * r
                rho = rho_new
    return s


# ---------------------------------------------------------------------------
# Givens-rotation GMRES building blocks
# ---------------------------------------------------------------------------

def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(apply_A, b, mask, tol, maxit, precond=None, restart=None, tol_abs=None):
    """(F)GMRES with x0 = 0 and modified Gram-Schmidt Arnoldi.
    precond=None: plain GMRES; otherwise right-preconditioned flexible GMRES
    (z_j = M v_j is stored, x = x0 + Z y).  Stops when the Givens residual
    estimate is <= tol * ||b|| (or <= tol_abs when given) or after maxit
    iterations; restart=None means unrestarted.
    Returns (x, iterations, final residual estimate)."""
    x = np.zeros_like(b)
    beta0 = norm_i(b, mask)
    target = tol_abs if tol_abs is not None else tol * beta0
    if beta0 == 0.0 or beta0 <= target:
        return x, 0, beta0
    m = restart if restart is not None else maxit
    total = 0
    r = np.where(mask, b, 0.0)
    res = beta0
    while True:
        beta = norm_i(r, mask)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        g[0] = beta
        cs = np.zeros(m)
        sn = np.zeros(m)
        k = 0
        for j in range(m):
            z = V[j] if precond is None else precond(V[j])
            Z.append(z)
            w = np.where(mask, apply_A(z), 0.0)
            for i in range(j + 1):
                H[i, j] = float(np.sum(w[mask] * V[i][mask]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = norm_i(w, mask)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            res = abs(g[j + 1])
            k = j + 1
            total += 1
            hnext = norm_i(w, mask)
            if res <= target or total >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        if res <= target or total >= maxit:
            return x, total, res
        r = np.where(mask, b - apply_A(x), 0.0)


# ---------------------------------------------------------------------------
# Algorithm 1: Jacobian-free multigrid V(nu1, nu2)-cycle
# ---------------------------------------------------------------------------

def mg_vcycle(levels, l, b, opts):
    """s_l = MG(x_l, F(x_l), b_l, l).  x_l, F(x_l) and lambda_l are taken from the
    levels (set once per Newton step by setup_levels)."""
    lv = levels[l]
    mode = opts.eps_mode_pc
    s = np.zeros(lv.shape)
    if l != 0:
        s = chebyshev(lv, s, lv.x, lv.Fx, b, opts.nu_pre, opts.cheb_degree, lv.lam_max,
                      opts.cheb_lo, opts.cheb_hi, mode)
        r = np.where(lv.mask, b - fd_jv(lv, lv.x, lv.Fx, s, mode), 0.0)
        r_c = transfer.restrict(r)
        c = mg_vcycle(levels, l - 1, r_c, opts)
        s = s + transfer.prolong(c)
        s = chebyshev(lv, s, lv.x, lv.Fx, b, opts.nu_post, opts.cheb_degree, lv.lam_max,
                      opts.cheb_lo, opts.cheb_hi, mode)
    else:
        maxit = opts.coarse_maxit if opts.coarse_maxit > 0 else lv.n_unknowns
        tol_abs = opts.coarse_tol if opts.coarse_tol_mode == "absolute" else None
        s, _, _ = gmres(lambda v: fd_jv(lv, lv.x, lv.Fx, v, mode), b, lv.mask,
                        opts.coarse_tol, maxit, tol_abs=tol_abs)
    return s


def setup_levels(levels, u, opts, newton_step):
    """Per Newton step: x_L = u, x_(l-1) = P x_l, F(x_l), and lambda_l by the
    power method on every level with a smoother (l >= 1)."""
    L = len(levels) - 1
    levels[L].x = u
    for l in range(L, 0, -1):
        levels[l - 1].x = transfer.project(levels[l].x)
    for l in range(L + 1):
        lv = levels[l]
        lv.Fx = lv.F(lv.x)
    for l in range(1, L + 1):
        lv = levels[l]
        if newton_step == 0 or lv.power_v is None:
            v0 = start_vector(lv.shape, opts.seed, l)
        else:
            v0 = lv.power_v
        lv.lam_max, lv.power_v = power_method(lv, lv.x, lv.Fx, v0, opts.power_iters,
                                              opts.eps_mode_pc, opts.power_tol)


# ---------------------------------------------------------------------------
# Line search and inexact Newton (Sec. 1 and Sec. 3 "Setup")
# ---------------------------------------------------------------------------

def backtrack(F_of, u, du, Fu, slope, c=1e-4, max_steps=10):
    """Backtracking on phi(alpha) = 1/2||F(u + alpha du)||^2 with quadratic and
    cubic interpolation.  Returns (alpha, F(u + alpha du), ok)."""
    f0 = 0.5 * float(np.sum(Fu * Fu))
    alpha = 1.0
    prev_alpha = prev_f = None
    for _ in range(max_steps):
        Fn = F_of(u + alpha * du)
        fn = 0.5 * float(np.sum(Fn * Fn))
        if fn <= f0 + c * alpha * slope:
            return alpha, Fn, True
        if prev_alpha is None:
            t = -slope * alpha * alpha / (2.0 * (fn - f0 - slope * alpha))
        else:
            r1 = fn - f0 - slope * alpha
            r2 = prev_f - f0 - slope * prev_alpha
            A = (r1 / alpha ** 2 - r2 / prev_alpha ** 2) / (alpha - prev_alpha)
            B = (-prev_alpha * r1 / alpha ** 2 + alpha * r2 / prev_alpha ** 2) / (alpha - prev_alpha)
            if A == 0.0:
                t = -slope / (2.0 * B)
            else:
                disc = B * B - 3.0 * A * slope
                t = (-B + np.sqrt(disc)) / (3.0 * A) if disc >= 0.0 else 0.5 * alpha
        t = min(max(t, 0.1 * alpha), 0.5 * alpha)
        prev_alpha, prev_f = alpha, fn
        alpha = t
    return alpha, Fn, False


@dataclass
class Stats:
    newton_its: int = 0
    linear_its: int = 0
    res_hist: list = field(default_factory=list)
    alpha_hist: list = field(default_factory=list)
    lin_hist: list = field(default_factory=list)
    lam_hist: list = field(default_factory=list)
    ge: float = 0.0
    converged: bool = False
    status: str = "ok"


def newton_solve(levels, u0, opts):
    """Inexact JFNK: x^(k+1) = x^(k) + alpha dx^(k), J dx = -F by MG-preconditioned
    FGMRES to ||J dx + F|| <= eta ||F||.  Returns (u, Stats)."""
    L = len(levels) - 1
    fine = levels[L]
    st = Stats()
    u = u0.copy()
    F = fine.F(u)
    F0 = norm_i(F, fine.mask)
    normF = F0
    st.res_hist.append(normF)
    for k in range(opts.max_newton):
        if F0 == 0.0 or normF <= opts.rtol_newton * F0 or (opts.atol_newton > 0 and normF < opts.atol_newton):
            st.converged = True
            break
        setup_levels(levels, u, opts, k)
        st.lam_hist.append([lv.lam_max for lv in levels[1:]])
        if opts.eta_mode == "paper":
            eta = min(opts.eta_max, normF)
        else:
            eta = min(opts.eta_max, normF / F0)
        Fx = F
        du, its, _ = gmres(lambda v: fd_jv(fine, u, Fx, v, "paper"), -F, fine.mask, eta,
                           opts.max_linear, precond=lambda v: mg_vcycle(levels, L, v, opts),
                           restart=opts.restart)
        st.linear_its += its
        st.lin_hist.append(its)
        if opts.line_search:
            slope = float(np.sum(F[fine.mask] * fd_jv(fine, u, F, du, "paper")[fine.mask]))
            alpha, Fn, ok = backtrack(fine.F, u, du, F, slope, max_steps=opts.ls_max)
            if not ok:
                st.status = "linesearch"
        else:
            alpha, Fn = 1.0, fine.F(u + du)
        u = u + alpha * du
        F = Fn
        normF = norm_i(F, fine.mask)
        st.res_hist.append(normF)
        st.alpha_hist.append(alpha)
        st.newton_its = k + 1
        if not np.isfinite(normF):
            st.status = "nonfinite"
            break
    else:
        st.converged = normF <= opts.rtol_newton * F0
    if normF <= opts.rtol_newton * F0:
        st.converged = True
    st.ge = total_ge(levels)
    return u, st
