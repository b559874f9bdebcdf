"""Q1 finite-element discretisation of the paper's nonlinear problems (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Conventions (readings of the paper, which fixes only "first order FE", Sec. 3):
  * Domain (0,1)^d, uniform grid of N elements per direction, h = 1/N,
    tensor-product Q1 elements on the structured grid.
  * Nodal arrays hold the FULL node grid including Dirichlet boundary nodes,
    shape (N+1,)*d with axis order (y, x) in 2D and (z, y, x) in 3D (x fastest).
    Boundary entries of u are the Dirichlet data; F is identically 0 there.
  * Element integrals use the 2^d-point tensor Gauss-Legendre rule with points
    1/2 +- 1/(2 sqrt 3) per direction and weights 1/2 (on [0,1]); it integrates
    the Q1 stiffness and mass exactly.  The nonlinear coefficients are evaluated
    at the Gauss points from u_h.
  * Per-element coefficient arrays (kappa) have shape (N,)*d, same axis order.

Problems:
  bratu2d  F_i = int grad u_h . grad phi_i - lam exp(u_h) phi_i      (Sec. 3, "Bratu":
           the gradient of Psi_B = int 1/2|grad u|^2 - lam exp(u); F = grad Psi, Sec. 1)
  nd3d     F_i = int (1+u_h^2) grad u_h . grad phi_i - b_i,  b_i = int f phi_i
           (nonlinear diffusion -div((1+u^2) grad u) = f, manufactured from
           u* = sin(pi x) sin(pi y) sin(pi z))
  ndk3d    F_i = sum_e kappa_e int_e (1+u_h^2) grad u_h . grad phi_i - int 1 phi_i
  minsurf2d F_i = int grad u_h . grad phi_i / sqrt(1 + |grad u_h|^2)   (Sec. 3, "Minimal
           Surface": the gradient of Psi_M = int sqrt(1 + |grad u|^2)); Dirichlet data
           u = 0 on x = 0 and x = 1, u = x(1-x) on y = 0 and y = 1 (minsurf_boundary)
"""
import itertools

import numpy as np
import scipy.sparse as sp

GAUSS_A = 1.0 / np.sqrt(3.0)
# 2-point Gauss-Legendre rule on [0, 1]
QP1 = np.array([0.5 - 0.5 * GAUSS_A, 0.5 + 0.5 * GAUSS_A])
QW1 = np.array([0.5, 0.5])
# 3-point Gauss-Legendre rule on [0, 1] (load vector only; f is not polynomial)
QP3 = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
QW3 = np.array([5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0])

KINDS = ("bratu2d", "nd3d", "ndk3d", "minsurf2d")


def dim_of(kind):
    """Spatial dimension of a problem kind (Sec. 3: Bratu and the minimal
    surface are 2D, nonlinear diffusion 3D)."""
    return 2 if kind in ("bratu2d", "minsurf2d") else 3


def local_nodes(d):
    """Local node offsets of a Q1 element, as tuples (ox, oy[, oz])."""
    return list(itertools.product((0, 1), repeat=d))


def shape1(o, xi):
    """1D linear shape function attached to local offset o, at xi in [0,1]."""
    return 1.0 - xi if o == 0 else xi


def dshape1(o):
    """Derivative of shape1 with respect to the reference coordinate."""
    return -1.0 if o == 0 else 1.0


def phi(off, xi):
    """Q1 shape function of local node off at reference point xi (tuples, x first)."""
    v = 1.0
    for o, x in zip(off, xi):
        v *= shape1(o, x)
    return v


def grad_phi(off, xi, h):
    """Physical gradient (x, y[, z]) of the Q1 shape function at reference point xi."""
    d = len(off)
    g = []
    for k in range(d):
        v = dshape1(off[k]) / h
        for m in range(d):
            if m != k:
                v *= shape1(off[m], xi[m])
        g.append(v)
    return g


def gauss_points(d, rule=2):
    """(reference point tuple x-first, weight on the unit cell) of the tensor rule."""
    p1, w1 = (QP1, QW1) if rule == 2 else (QP3, QW3)
    out = []
    for idx in itertools.product(range(len(p1)), repeat=d):
        out.append((tuple(p1[i] for i in idx), float(np.prod([w1[i] for i in idx]))))
    return out


def _slices(off, n):
    """Array slice selecting, for every element, the node at local offset off.
    Array axes are reversed relative to the offset tuple (x is the last axis)."""
    return tuple(slice(o, o + n) for o in reversed(off))


def gather_element_values(u):
    """Dict local-offset -> array over all elements of the nodal value there."""
    d = u.ndim
    n = u.shape[0] - 1
    return {off: u[_slices(off, n)] for off in local_nodes(d)}


def scatter_add(F, contrib):
    """Add per-element local contributions into the global nodal array."""
    n = F.shape[0] - 1
    for off, c in contrib.items():
        F[_slices(off, n)] += c
    return F


def boundary_mask(shape):
    """Boolean array, True on Dirichlet boundary nodes."""
    m = np.zeros(shape, dtype=bool)
    for ax in range(len(shape)):
        sl = [slice(None)] * len(shape)
        sl[ax] = 0
        m[tuple(sl)] = True
        sl[ax] = -1
        m[tuple(sl)] = True
    return m


def interior(shape):
    """True at the unknowns: every node not on the Dirichlet boundary."""
    return ~boundary_mask(shape)


# ---------------------------------------------------------------------------
# Element routine: local residual contributions of every element
# ---------------------------------------------------------------------------

def element_residual(kind, U, h, lam=0.0, kappa=None):
    """Local contributions  int_e  flux(u_h) . grad phi_a  (+ source)  for every element.

    U: dict offset -> array over elements of nodal values.  Returns dict offset ->
    array.  The Gauss rule is applied exactly as written in the module docstring:
    u_h and grad u_h at each point, the pointwise nonlinearity, then the test
    functions.
    """
    d = dim_of(kind)
    offs = local_nodes(d)
    shape = next(iter(U.values())).shape
    C = {off: np.zeros(shape) for off in offs}
    vol = h ** d
    for xi, w in gauss_points(d):
        uq = np.zeros(shape)
        gq = [np.zeros(shape) for _ in range(d)]
        for off in offs:
            ph = phi(off, xi)
            gp = grad_phi(off, xi, h)
            uq += ph * U[off]
            for k in range(d):
                gq[k] += gp[k] * U[off]
        if kind == "bratu2d":
            coef = 1.0
            src = -lam * np.exp(uq)
        elif kind == "minsurf2d":
            coef = 1.0 / np.sqrt(1.0 + sum(g * g for g in gq))
            src = None
        else:
            coef = 1.0 + uq * uq
            if kind == "ndk3d":
                coef = coef * kappa
            src = None
        for off in offs:
            gp = grad_phi(off, xi, h)
            val = coef * sum(gq[k] * gp[k] for k in range(d))
            if src is not None:
                val = val + src * phi(off, xi)
            C[off] += w * vol * val
    return C


def operator(kind, u, lam=0.0, kappa=None):
    """A(u): the residual without the constant load term, boundary rows zero."""
    d = u.ndim
    assert d == dim_of(kind)
    n = u.shape[0] - 1
    h = 1.0 / n
    U = gather_element_values(u)
    F = scatter_add(np.zeros(u.shape), element_residual(kind, U, h, lam, kappa))
    F[boundary_mask(u.shape)] = 0.0
    return F


def unit_load(shape):
    """int 1 * phi_i on interior nodes (the ND-kappa source), zero on the boundary.
    Evaluated with the same Gauss rule (exact for Q1)."""
    d = len(shape)
    n = shape[0] - 1
    h = 1.0 / n
    C = {}
    for off in local_nodes(d):
        C[off] = np.full((n,) * d, sum(w * phi(off, xi) for xi, w in gauss_points(d)) * h ** d)
    b = scatter_add(np.zeros(shape), C)
    b[boundary_mask(shape)] = 0.0
    return b


def residual(kind, u, lam=0.0, kappa=None, load=None):
    """F(u) of the chosen problem (Sec. 1: F = grad Psi for Bratu; Sec. 3 problems).

    load: for nd3d the vector b_i = int f phi_i (see mms_load); ignored otherwise.
    """
    F = operator(kind, u, lam, kappa)
    if kind == "nd3d" and load is not None:
        F = F - load
    elif kind == "ndk3d":
        F = F - unit_load(u.shape)
    F[boundary_mask(u.shape)] = 0.0
    return F


def bratu_energy(u, lam):
    """Discrete Bratu energy Psi_B(u_h) = int 1/2|grad u_h|^2 - lam exp(u_h) with the
    same Gauss rule (Sec. 3, Bratu).  Its gradient with respect to the interior
    nodal values is F (Sec. 1: F = grad Psi)."""
    n = u.shape[0] - 1
    h = 1.0 / n
    U = gather_element_values(u)
    shape = next(iter(U.values())).shape
    E = np.zeros(shape)
    for xi, w in gauss_points(2):
        uq = sum(phi(off, xi) * U[off] for off in U)
        g = [sum(grad_phi(off, xi, h)[k] * U[off] for off in U) for k in range(2)]
        E += w * h * h * (0.5 * (g[0] ** 2 + g[1] ** 2) - lam * np.exp(uq))
    return float(E.sum())


def minsurf_energy(u):
    """Discrete area Psi_M(u_h) = int sqrt(1 + |grad u_h|^2) with the same Gauss
    rule (Sec. 3, minimal surface); its gradient with respect to the interior
    nodal values is F."""
    n = u.shape[0] - 1
    h = 1.0 / n
    U = gather_element_values(u)
    shape = next(iter(U.values())).shape
    E = np.zeros(shape)
    for xi, w in gauss_points(2):
        g = [sum(grad_phi(off, xi, h)[k] * U[off] for off in U) for k in range(2)]
        E += w * h * h * np.sqrt(1.0 + g[0] ** 2 + g[1] ** 2)
    return float(E.sum())


def minsurf_boundary(n):
    """Node grid with the Dirichlet data of the minimal-surface example (Sec. 3):
    u = x(1-x) on the edges y = 0 and y = 1, u = 0 on x = 0 and x = 1; interior 0."""
    u = np.zeros((n + 1, n + 1))
    x = np.linspace(0.0, 1.0, n + 1)
    u[0, :] = x * (1.0 - x)
    u[-1, :] = x * (1.0 - x)
    return u


# ---------------------------------------------------------------------------
# Manufactured load for nd3d
# ---------------------------------------------------------------------------

def mms_exact(x, y, z):
    """u* = sin(pi x) sin(pi y) sin(pi z)."""
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def mms_source(x, y, z):
    """f = -div((1+u*^2) grad u*) for u* = sin(pi x) sin(pi y) sin(pi z), in closed form:
    f = (1+u*^2) 3 pi^2 u* - 2 u* |grad u*|^2."""
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
    u = sx * sy * sz
    g2 = np.pi ** 2 * ((cx * sy * sz) ** 2 + (sx * cy * sz) ** 2 + (sx * sy * cz) ** 2)
    return (1.0 + u * u) * 3.0 * np.pi ** 2 * u - 2.0 * u * g2


def mms_load(n):
    """b_i = int f phi_i over the grid of n elements per direction, 3-point Gauss
    rule per direction (f is not polynomial), zero on boundary nodes."""
    h = 1.0 / n
    e = np.arange(n) * h
    ez, ey, ex = np.meshgrid(e, e, e, indexing="ij")
    C = {off: np.zeros((n, n, n)) for off in local_nodes(3)}
    for xi, w in gauss_points(3, rule=3):
        fq = mms_source(ex + xi[0] * h, ey + xi[1] * h, ez + xi[2] * h)
        for off in C:
            C[off] += w * h ** 3 * fq * phi(off, xi)
    b = scatter_add(np.zeros((n + 1,) * 3), C)
    b[boundary_mask(b.shape)] = 0.0
    return b


def mms_load_at(n, nodes):
    """b_i of mms_load at the given interior nodes only (array-order index
    tuples): the same 3-point rule on the 8 elements around each node."""
    h = 1.0 / n
    out = []
    for node in nodes:
        k, j, i = (int(t) for t in node)
        if min(i, j, k) == 0 or max(i, j, k) == n:
            out.append(0.0)
            continue
        total = 0.0
        for ez in (k - 1, k):
            for ey in (j - 1, j):
                for ex in (i - 1, i):
                    loc = (i - ex, j - ey, k - ez)  # x-first local offset of the node
                    for xi, w in gauss_points(3, rule=3):
                        fq = mms_source((ex + xi[0]) * h, (ey + xi[1]) * h, (ez + xi[2]) * h)
                        total += w * h ** 3 * fq * phi(loc, xi)
        out.append(total)
    return np.array(out)


def node_coords(n, d):
    """Coordinate arrays (x, y[, z]) of the full node grid, in array axis order."""
    t = np.linspace(0.0, 1.0, n + 1)
    grids = np.meshgrid(*([t] * d), indexing="ij")
    return tuple(reversed(grids))  # (x, y[, z]) with x along the last axis


# ---------------------------------------------------------------------------
# Residual at a few sampled nodes (for checks at sizes where a full oracle
# evaluation is too slow).  Same element routine, applied to the 2^d elements
# around each sampled node.
# ---------------------------------------------------------------------------

def residual_at(kind, u, nodes, lam=0.0, kappa=None, load=None):
    """F at the given interior nodes (list of index tuples in array axis order)."""
    d = u.ndim
    n = u.shape[0] - 1
    h = 1.0 / n
    out = []
    for node in nodes:
        node = tuple(int(t) for t in node)
        if any(t == 0 or t == n for t in node):
            out.append(0.0)
            continue
        total = 0.0
        # elements whose lower corner is node - o for o in {0,1}^d (array order)
        for eo in itertools.product((0, 1), repeat=d):
            ecorner = tuple(node[a] - eo[a] for a in range(d))
            U = {}
            for off in local_nodes(d):
                idx = tuple(ecorner[a] + off[d - 1 - a] for a in range(d))
                U[off] = np.array([u[idx]])
            kap = None
            if kappa is not None:
                kap = np.array([kappa[ecorner]])
            C = element_residual(kind, U, h, lam, kap)
            # local offset of the node inside this element, x first
            loc = tuple(reversed(eo))
            total += float(C[loc][0])
        if kind == "nd3d" and load is not None:
            total -= float(load[node])
        elif kind == "ndk3d":
            total -= h ** d
        out.append(total)
    return np.array(out)


# ---------------------------------------------------------------------------
# Analytic Jacobian, assembled (for pins only; the method never assembles it)
# ---------------------------------------------------------------------------

def _global_index(shape, arr_idx):
    return np.ravel_multi_index(arr_idx, shape)


def assemble_jacobian(kind, u, lam=0.0, kappa=None):
    """Sparse dF/du on the full node numbering, with boundary rows and columns
    replaced by zero (the unknowns are the interior nodes).  Written from the
    derivative of the element integrand:
      bratu2d  J_ab = int grad phi_b . grad phi_a - lam exp(u_h) phi_b phi_a
      minsurf2d J_ab = int grad phi_b . grad phi_a / q - (grad u_h . grad phi_a)(grad u_h . grad phi_b) / q^3,
               q = sqrt(1 + |grad u_h|^2)
      nd3d     J_ab = int (1+u_h^2) grad phi_b . grad phi_a + 2 u_h phi_b grad u_h . grad phi_a
      ndk3d    kappa_e times the nd3d integrand.
    """
    d = u.ndim
    n = u.shape[0] - 1
    h = 1.0 / n
    offs = local_nodes(d)
    U = gather_element_values(u)
    eshape = (n,) * d
    Ke = {(a, b): np.zeros(eshape) for a in offs for b in offs}
    for xi, w in gauss_points(d):
        uq = sum(phi(off, xi) * U[off] for off in offs)
        gq = [sum(grad_phi(off, xi, h)[k] * U[off] for off in offs) for k in range(d)]
        for a in offs:
            ga = grad_phi(a, xi, h)
            pa = phi(a, xi)
            for b in offs:
                gb = grad_phi(b, xi, h)
                pb = phi(b, xi)
                gab = sum(ga[k] * gb[k] for k in range(d))
                if kind == "bratu2d":
                    val = gab - lam * np.exp(uq) * pb * pa
                elif kind == "minsurf2d":
                    q2 = 1.0 + sum(gq[k] * gq[k] for k in range(d))
                    gua = sum(gq[k] * ga[k] for k in range(d))
                    gub = sum(gq[k] * gb[k] for k in range(d))
                    val = gab / np.sqrt(q2) - gua * gub / q2 ** 1.5
                else:
                    val = (1.0 + uq * uq) * gab + 2.0 * uq * pb * sum(gq[k] * ga[k] for k in range(d))
                    if kind == "ndk3d":
                        val = val * kappa
                Ke[(a, b)] += w * h ** d * val
    grid = np.indices(eshape)  # array-order element corner indices
    rows, cols, vals = [], [], []
    for a in offs:
        ia = tuple(grid[ax] + a[d - 1 - ax] for ax in range(d))
        ga_idx = _global_index(u.shape, ia).ravel()
        for b in offs:
            ib = tuple(grid[ax] + b[d - 1 - ax] for ax in range(d))
            gb_idx = _global_index(u.shape, ib).ravel()
            rows.append(ga_idx)
            cols.append(gb_idx)
            vals.append(Ke[(a, b)].ravel())
    N = u.size
    J = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    keep = interior(u.shape).ravel().astype(float)
    Dk = sp.diags(keep)
    return (Dk @ J @ Dk).tocsr()


# ---------------------------------------------------------------------------
# Vector-Jacobian products for the coefficient problem (adjoint pattern)
# ---------------------------------------------------------------------------

def vjp_ndk3d(u, kappa, w):
    """J(u)^T w and (dF/dkappa)^T w for ndk3d, element by element.

    (J^T w)_b = sum_e kappa_e int_e (1+u_h^2) grad phi_b . grad w_h + 2 u_h phi_b grad u_h . grad w_h
    (dF/dkappa_e)^T w = int_e (1+u_h^2) grad u_h . grad w_h
    w is restricted to interior nodes first (boundary rows of F are not equations);
    J^T w is zero on boundary nodes (boundary values are not unknowns).
    """
    d = 3
    n = u.shape[0] - 1
    h = 1.0 / n
    offs = local_nodes(d)
    wi = np.where(interior(u.shape), w, 0.0)
    U = gather_element_values(u)
    W = gather_element_values(wi)
    eshape = (n,) * d
    C = {off: np.zeros(eshape) for off in offs}
    dk = np.zeros(eshape)
    for xi, wq in gauss_points(d):
        uq = sum(phi(off, xi) * U[off] for off in offs)
        gu = [sum(grad_phi(off, xi, h)[k] * U[off] for off in offs) for k in range(d)]
        gw = [sum(grad_phi(off, xi, h)[k] * W[off] for off in offs) for k in range(d)]
        gugw = sum(gu[k] * gw[k] for k in range(d))
        dk += wq * h ** d * (1.0 + uq * uq) * gugw
        for b in offs:
            gb = grad_phi(b, xi, h)
            val = (1.0 + uq * uq) * sum(gb[k] * gw[k] for k in range(d)) + 2.0 * uq * phi(b, xi) * gugw
            C[b] += wq * h ** d * kappa * val
    JTw = scatter_add(np.zeros(u.shape), C)
    JTw[boundary_mask(u.shape)] = 0.0
    return JTw, dk
