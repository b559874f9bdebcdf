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

Readings (where the paper is silent, or where the default settings differ from it):
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
  * Coarse solve: unrestarted GMRES (the default settings use GMRES where
    the paper uses CG), x0 = 0, modified Gram-Schmidt, stop at
    ||r|| <= tol ||r_0|| (relative reading) or after n_0 iterations.
  * Outer Krylov: right-preconditioned flexible GMRES(m) (the default
    settings; the paper uses CG because its J is symmetric, see pcg).
  * Forcing term: eta = min(0.5, ||F_k|| / ||F_0||) (relative reading of
    eta = min(0.5, ||F||)); the paper's absolute form is an option.
  * Line search: backtracking with quadratic then cubic interpolation
    (Dennis & Schnabel, Numerical Methods for Unconstrained Optimization and
    Nonlinear Equations, Sec. 6.3) on phi(alpha) = 1/2 ||F(u + alpha dx)||^2,
    Armijo constant 1e-4, new step clipped to [0.1, 0.5] alpha, at most 10
    residual evaluations; without sufficient decrease the step is not taken
    and the solve stops.  The slope phi'(0) = F . (J dx): after a single
    FGMRES cycle from the Arnoldi relation of that cycle (the FD actions it
    already applied), otherwise (restarts, CG) from one more FD action.
  * P x^(k) and F(P x^(k)) on each level are evaluated once per Newton step
    (x^(k) does not change during the step, so this equals re-evaluating
    them inside every cycle as Alg. 1 writes it).

The paper's own solver variant (``paper_options``): CG outer Krylov method,
coarse CG preconditioned by L-BFGS with the spectral shift of Alg. 1.  Its
readings:
  * "V(5,5)" = one application of the degree-5 Chebyshev polynomial per side
    (one recurrence step per smoothing step).
  * Outer CG, negative curvature p.Jp <= 0: stop and return the current
    iterate, or the first search direction when it happens at the first
    iteration (Nocedal & Wright, Numerical Optimization, 2nd ed., Alg. 7.1).
  * Coarse CG: stop at ||r|| <= tol ||b|| (relative reading, as for GMRES) or
    after n_0 iterations per call; on negative curvature return the current
    iterate and lambda_c = p.A_s p / p.p of the operator CG is applied to,
    A_s = A - lambda_c+ I (lambda_c+ <= 0); a call without negative curvature
    returns lambda_c = 0.  A shifted call restarts CG from the returned s_0.
  * Secant pairs (Morales & Nocedal, SIAM J. Optim. 10 (2000)): during the very
    first coarse CG call every step gives s_i = alpha_i p_i, y_i = alpha_i A p_i;
    after that call m of the k pairs are kept, those of iterations
    floor(j k / m), j = 0..m-1 (all of them when k <= m) -- "uniform sampling".
    The preconditioner is the L-BFGS inverse-Hessian approximation applied by
    the two-loop recursion (Nocedal & Wright, Alg. 7.4) with
    H_0 = (s^T y / y^T y) I of the last kept pair; it is kept for the rest of
    the solve.
  * At most 30 shifted calls per coarse solve (the shift grows at least by the
    factor gamma per call).
"""
from dataclasses import dataclass, field

import numpy as np

from . import fem, hyper, transfer
from .splitmix import start_vector

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


@dataclass
class Options:
    """Solver settings; the defaults are the 2D Bratu workload's (V(3,3),
    degree 3 on [0.1, 1.1] lambda, 10 power iterations, FGMRES(30)) and
    paper_options() gives the paper's own (Sec. 2, Sec. 3 "Setup")."""
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
    outer: str = "fgmres"           # or "cg" (the paper's outer method)
    coarse: str = "gmres"           # or "cgqn" (the paper's coarse solver)
    lbfgs_pairs: int = 20
    shift_gamma: float = 5.0


def paper_options(**kw):
    """The paper's own settings (Sec. 2 and Sec. 3 "Setup"): CG preconditioned by
    the V(5,5) cycle, Chebyshev on [0.06, 1.2] lambda_l, power method to 30
    iterations or a change below 1e-2, coarse CG with 20 L-BFGS secant pairs and
    the spectral shift gamma = 5, eta = min(0.5, ||F||), stop at ||F|| < 1e-6."""
    o = Options(nu_pre=1, nu_post=1, cheb_degree=5, cheb_lo=0.06, cheb_hi=1.2, power_iters=30,
                power_tol=1e-2, rtol_newton=0.0, atol_newton=1e-6, eta_mode="paper", outer="cg",
                coarse="cgqn", lbfgs_pairs=20, shift_gamma=5.0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# Level hierarchy {T_l}, l = 0 (coarsest) .. L (finest)   (Sec. 2)
# ---------------------------------------------------------------------------

class Level:
    """One level of the hierarchy (Sec. 2): the rediscretised operator on n
    elements per direction, its current iterate x, F(x) and lambda_max."""

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
        self.lbfgs = None    # coarse level: L-BFGS preconditioner of the first coarse CG call

    def F(self, x):
        self.ge += 1
        return fem.residual(self.kind, x, self.lam, self.kappa, self.load)

    # transfers to and from the next coarser level (Sec. 2)
    def restrict(self, r):
        return transfer.restrict(r)

    def prolong(self, c):
        return transfer.prolong(c)

    def project(self, x):
        return transfer.project(x)


class HyperLevel(Level):
    """A level of the hyperelastic beam (Sec. 3): 10m x m x m elements, three
    displacement components per node, unknowns away from x = 0 and x = 10."""

    def __init__(self, m):
        self.kind = "hyper3d"
        self.n = m
        self.d = 3
        self.lam = 0.0
        self.kappa = None
        self.load = None
        self.shape = hyper.shape_of(m)
        self.mask = hyper.unknown_mask(self.shape)
        self.n_unknowns = int(self.mask.sum())
        self.ge = 0
        self.x = None
        self.Fx = None
        self.lam_max = None
        self.power_v = None
        self.lbfgs = None

    def F(self, x):
        self.ge += 1
        return hyper.residual(x)

    def restrict(self, r):
        return hyper.restrict(r)

    def prolong(self, c):
        return hyper.prolong(c)

    def project(self, x):
        return hyper.project(x)


def build_hyper_hierarchy(k):
    """Levels l = 0..k of the beam at refinement level L_k: m_l = 2^l (T_0 = 10 x 1 x 1)."""
    return [HyperLevel(2 ** l) for l in range(k + 1)]


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
    """Euclidean norm over the unknowns."""
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


def gmres(apply_A, b, mask, tol, maxit, precond=None, restart=None, tol_abs=None, info=None):
    """(F)GMRES with x0 = 0 and modified Gram-Schmidt Arnoldi.
    precond=None: plain GMRES; otherwise right-preconditioned flexible GMRES
    (z_j = M v_j is stored, x = x0 + Z y).  Stops when the Givens residual
    estimate is <= tol * ||b|| (or <= tol_abs when given) or after maxit
    iterations; restart=None means unrestarted.
    Returns (x, iterations, final residual estimate).

    info (a dict, optional) receives "cycles" (Arnoldi cycles run) and, from
    the last cycle, "beta" = ||r|| at its start and "Hy0" = (Hbar y)_0, the
    first entry of the unrotated (k+1) x k Hessenberg matrix times the
    least-squares solution.  With one cycle (x0 = 0, v_0 = b / beta) the
    Arnoldi relation A Z y = V_(k+1) Hbar y gives b . (A x) = beta Hy0 from the
    actions already applied."""
    x = np.zeros_like(b)
    beta0 = norm_i(b, mask)
    target = tol_abs if tol_abs is not None else tol * beta0
    if info is not None:
        info.update(cycles=0, beta=beta0, Hy0=0.0)
    if beta0 == 0.0 or beta0 <= target:
        return x, 0, beta0
    m = restart if restart is not None else maxit
    total = 0
    r = np.where(mask, b, 0.0)
    res = beta0
    cycles = 0
    while True:
        cycles += 1
        beta = norm_i(r, mask)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        Hraw = np.zeros((m + 1, m))
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
            Hraw[:j + 2, j] = H[:j + 2, j]
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
        if info is not None:
            info.update(cycles=cycles, beta=beta, Hy0=float(np.dot(Hraw[0, :k], y)))
        if res <= target or total >= maxit:
            return x, total, res
        r = np.where(mask, b - apply_A(x), 0.0)


# ---------------------------------------------------------------------------
# Conjugate gradients, L-BFGS preconditioner, shifted coarse CG
# (Sec. 2 "The coarse level solver", Alg. 1, Sec. 3 "Setup")
# ---------------------------------------------------------------------------

def _dot(a, b, mask):
    return float(np.sum(a[mask] * b[mask]))


def pcg(apply_A, b, mask, tol, maxit, precond=None, tol_abs=None):
    """Preconditioned CG for A x = b from x0 = 0 (the paper's outer Krylov method).
    Stops at ||r|| <= tol ||b|| (or tol_abs) or after maxit iterations.  On
    negative curvature p.Ap <= 0 it stops and returns the current iterate, or
    the first search direction if that happens at the first iteration.
    Returns (x, iterations, ||r||, negative_curvature)."""
    x = np.zeros_like(b)
    r = np.where(mask, b, 0.0)
    res = norm_i(r, mask)
    target = tol_abs if tol_abs is not None else tol * res
    if res == 0.0 or res <= target:
        return x, 0, res, False
    z = np.where(mask, r if precond is None else precond(r), 0.0)
    p = z
    rz = _dot(r, z, mask)
    for it in range(1, maxit + 1):
        q = np.where(mask, apply_A(p), 0.0)
        pq = _dot(p, q, mask)
        if pq <= 0.0:
            return (p if it == 1 else x), it, res, True
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        res = norm_i(r, mask)
        if res <= target:
            return x, it, res, False
        z = np.where(mask, r if precond is None else precond(r), 0.0)
        rz_new = _dot(r, z, mask)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, res, False


class LBFGS:
    """L-BFGS inverse-Hessian approximation H from secant pairs (s_i, y_i), oldest
    first, applied by the two-loop recursion (Nocedal & Wright, Alg. 7.4) with
    H_0 = gamma I, gamma = s^T y / y^T y of the last pair."""

    def __init__(self, pairs, mask):
        self.S = [p[0] for p in pairs]
        self.Y = [p[1] for p in pairs]
        self.mask = mask

    def apply(self, r):
        m = self.mask
        q = np.where(m, r, 0.0)
        k = len(self.S)
        if k == 0:
            return q
        rho = [1.0 / _dot(self.Y[i], self.S[i], m) for i in range(k)]
        a = [0.0] * k
        for i in range(k - 1, -1, -1):
            a[i] = rho[i] * _dot(self.S[i], q, m)
            q = q - a[i] * self.Y[i]
        gamma = _dot(self.S[-1], self.Y[-1], m) / _dot(self.Y[-1], self.Y[-1], m)
        z = gamma * q
        for i in range(k):
            bta = rho[i] * _dot(self.Y[i], z, m)
            z = z + (a[i] - bta) * self.S[i]
        return z


def uniform_sample(pairs, m):
    """Keep the pairs of iterations floor(j k / m), j = 0..m-1, of a run of k steps
    (all of them when k <= m)."""
    k = len(pairs)
    if k <= m:
        return list(pairs)
    return [pairs[(j * k) // m] for j in range(m)]


def coarse_cg(apply_A, b, mask, s0, shift, tol, maxit, H=None, collect=None, tol_abs=None):
    """CG(s_0, x_0, F(x_0), r_0, lambda_c+, nu_*) of Alg. 1: CG for
    (A - lambda_c+ I) s = b from s_0, preconditioned by the L-BFGS operator H when
    given.  Appends the secant pairs (alpha p, alpha A_s p) to ``collect`` when
    it is a list.  Returns (s, lambda_c, iterations): lambda_c is the Rayleigh
    quotient p.A_s p / p.p at negative curvature, else 0."""
    def A_s(v):
        return np.where(mask, apply_A(v) - shift * v, 0.0)

    x = np.where(mask, s0, 0.0)
    nb = norm_i(b, mask)
    target = tol_abs if tol_abs is not None else tol * nb
    r = np.where(mask, b, 0.0) - (A_s(x) if np.any(x[mask] != 0.0) else 0.0)
    res = norm_i(r, mask)
    if res == 0.0 or res <= target:
        return x, 0.0, 0
    z = H.apply(r) if H is not None else r
    p = z
    rz = _dot(r, z, mask)
    for it in range(1, maxit + 1):
        q = A_s(p)
        pq = _dot(p, q, mask)
        if pq <= 0.0:
            return x, pq / _dot(p, p, mask), it
        alpha = rz / pq
        if collect is not None:
            collect.append((alpha * p, alpha * q))
        x = x + alpha * p
        r = r - alpha * q
        res = norm_i(r, mask)
        if res <= target:
            return x, 0.0, it
        z = H.apply(r) if H is not None else r
        rz_new = _dot(r, z, mask)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, 0.0, maxit


def coarse_cgqn(apply_A, b, lv, tol, maxit, m, gamma, tol_abs=None, max_shifts=30):
    """Coarse branch of Alg. 1: lambda_c+ = 0; (s_0, lambda_c) = CG(...); while
    lambda_c < 0: lambda_c+ = gamma min(lambda_c, lambda_c+), (s_0, lambda_c) =
    CG(...) with the shifted operator.  The first call on this level collects the
    secant pairs of the L-BFGS preconditioner (kept in lv.lbfgs).
    Returns (s_0, list of the shifts lambda_c+ used)."""
    shift = 0.0
    collect = [] if lv.lbfgs is None else None
    s, lam_c, _ = coarse_cg(apply_A, b, lv.mask, np.zeros_like(b), shift, tol, maxit, lv.lbfgs, collect,
                            tol_abs)
    if collect is not None:
        lv.lbfgs = LBFGS(uniform_sample(collect, m), lv.mask)
    shifts = [shift]
    while lam_c < 0.0 and len(shifts) <= max_shifts:
        shift = gamma * min(lam_c, shift)
        shifts.append(shift)
        s, lam_c, _ = coarse_cg(apply_A, b, lv.mask, s, shift, tol, maxit, lv.lbfgs, None, tol_abs)
    return s, shifts


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
        r_c = lv.restrict(r)
        c = mg_vcycle(levels, l - 1, r_c, opts)
        s = s + lv.prolong(c)
        s = chebyshev(lv, s, lv.x, lv.Fx, b, opts.nu_post, opts.cheb_degree, lv.lam_max,
                      opts.cheb_lo, opts.cheb_hi, mode)
    else:
        maxit = opts.coarse_maxit if opts.coarse_maxit > 0 else lv.n_unknowns
        tol_abs = opts.coarse_tol if opts.coarse_tol_mode == "absolute" else None
        apply_A = lambda v: fd_jv(lv, lv.x, lv.Fx, v, mode)  # noqa: E731
        if opts.coarse == "cgqn":
            s, shifts = coarse_cgqn(apply_A, b, lv, opts.coarse_tol, maxit, opts.lbfgs_pairs,
                                    opts.shift_gamma, tol_abs=tol_abs)
            lv.shift_calls = getattr(lv, "shift_calls", 0) + len(shifts) - 1
        else:
            s, _, _ = gmres(apply_A, b, lv.mask, opts.coarse_tol, maxit, tol_abs=tol_abs)
    return s


def setup_levels(levels, u, opts, newton_step):
    """Per Newton step: x_L = u, x_(l-1) = P x_l, F(x_l), and lambda_l by the
    power method on every level with a smoother (l >= 1)."""
    L = len(levels) - 1
    levels[L].x = u
    for l in range(L, 0, -1):
        levels[l - 1].x = levels[l].project(levels[l].x)
    for l in range(L + 1):
        lv = levels[l]
        lv.Fx = lv.F(lv.x)
    for l in range(1, L + 1):
        lv = levels[l]
        if newton_step == 0 or lv.power_v is None:
            v0 = start_vector(lv.shape, opts.seed, l, lv.mask)
        else:
            v0 = lv.power_v
        lv.lam_max, lv.power_v = power_method(lv, lv.x, lv.Fx, v0, opts.power_iters,
                                              opts.eps_mode_pc, opts.power_tol)


# ---------------------------------------------------------------------------
# Line search and inexact Newton (Sec. 1 and Sec. 3 "Setup")
# ---------------------------------------------------------------------------

def backtrack(F_of, u, du, Fu, slope, c=1e-4, max_steps=10, trials=None):
    """Backtracking on phi(alpha) = 1/2||F(u + alpha du)||^2 with quadratic and
    cubic interpolation (Dennis & Schnabel, Sec. 6.3).

    The full step alpha = 1 is tried first.  A rejected trial is followed by the
    minimiser of the quadratic through phi(0), phi'(0) = slope and the trial,
    after that by the local minimiser of the cubic through phi(0), phi'(0) and
    the last two trials; the new step is clipped to [0.1, 0.5] alpha.  A trial
    whose residual is not finite (e.g. an inverted element of the hyperelastic
    beam, J <= 0) is cut to 0.1 alpha and not used as an interpolation point.
    At most max_steps residuals are evaluated.

    Returns (alpha, F(u + alpha du), ok): the accepted step, or, when no trial
    gave the sufficient decrease phi <= phi(0) + c alpha slope, the last
    tested step with its own residual and ok = False.  The tested steps are
    appended to `trials` when a list is given."""
    f0 = 0.5 * float(np.sum(Fu * Fu))
    alpha = 1.0
    prev_alpha = prev_f = None
    Fn = None
    tested = alpha
    for _ in range(max_steps):
        Fn = F_of(u + alpha * du)
        tested = alpha
        if trials is not None:
            trials.append(alpha)
        fn = 0.5 * float(np.sum(Fn * Fn))
        if fn <= f0 + c * alpha * slope:
            return alpha, Fn, True
        if not np.isfinite(fn):
            prev_alpha = prev_f = None
            alpha = 0.1 * alpha
            continue
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
    return tested, Fn, False


@dataclass
class Stats:
    """Counts of one Newton solve: iterations, residual history and GE (Sec. 3)."""
    newton_its: int = 0
    linear_its: int = 0
    res_hist: list = field(default_factory=list)
    alpha_hist: list = field(default_factory=list)
    ls_hist: list = field(default_factory=list)
    lin_hist: list = field(default_factory=list)
    lam_hist: list = field(default_factory=list)
    ge: float = 0.0
    converged: bool = False
    status: str = "ok"


def newton_solve(levels, u0, opts):
    """Inexact JFNK: x^(k+1) = x^(k) + alpha dx^(k), J dx = -F by MG-preconditioned
    FGMRES (or CG, the paper's choice) to ||J dx + F|| <= eta ||F||.
    Returns (u, Stats)."""
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
        if not np.isfinite(normF):
            st.status = "nonfinite"
            break
        setup_levels(levels, u, opts, k)
        st.lam_hist.append([lv.lam_max for lv in levels[1:]])
        if opts.eta_mode == "paper":
            eta = min(opts.eta_max, normF)
        else:
            eta = min(opts.eta_max, normF / F0)
        Fx = F
        apply_J = lambda v: fd_jv(fine, u, Fx, v, "paper")  # noqa: E731
        mg = lambda v: mg_vcycle(levels, L, v, opts)  # noqa: E731
        ginfo = {}
        if opts.outer == "cg":
            du, its, _, _ = pcg(apply_J, -F, fine.mask, eta, opts.max_linear, precond=mg)
        else:
            du, its, _ = gmres(apply_J, -F, fine.mask, eta, opts.max_linear, precond=mg,
                               restart=opts.restart, info=ginfo)
        st.linear_its += its
        st.lin_hist.append(its)
        if opts.line_search:
            if ginfo.get("cycles") == 1:
                # phi'(0) = F . (J du) from the Arnoldi relation of the single
                # FGMRES cycle: b = -F = beta v_0, so F . (J Z y) = -beta (Hbar y)_0
                slope = -ginfo["beta"] * ginfo["Hy0"]
            else:
                slope = float(np.sum(F[fine.mask] * fd_jv(fine, u, F, du, "paper")[fine.mask]))
            trials = []
            alpha, Fn, ok = backtrack(fine.F, u, du, F, slope, max_steps=opts.ls_max, trials=trials)
            st.ls_hist.append(len(trials))
            if not ok:
                # no sufficient decrease: the step is not taken and the solve
                # stops at the last accepted iterate (Dennis & Schnabel, Sec. 6.3)
                st.status = "linesearch"
                st.res_hist.append(normF)
                st.alpha_hist.append(0.0)
                st.newton_its = k + 1
                break
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
