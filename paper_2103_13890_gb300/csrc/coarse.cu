// Coarse-level solve of Algorithm 1 (l = 0): a matrix-free Krylov method in
// place of a direct solver (Sec. 2, "The coarse level solver").  The default
// settings use unrestarted GMRES with x0 = 0; it stops when the Givens
// residual estimate is <= tol ||r0|| (relative reading) or <= tol (absolute),
// or after maxit iterations (Sec. 3: maxit = number of coarse unknowns).
//
// The coarse grid is tiny (<= JFNK_COARSE_MAX_NODES nodes), so the whole
// solve runs in ONE CTA: the FD Jacobian action (element loop into shared
// memory, node gather), classical Gram-Schmidt applied twice, Givens rotations
// and the back-substitution, with no kernel launches or host round-trips.
#include "coarse.cuh"
#include "element.cuh"
#include "reduce.cuh"
#include "stencil.cuh"

namespace jfnk {

constexpr int kCoarseThreads = 512;

// Threads of the one-CTA coarse solvers: about one per node, in whole warps,
// 64 to 512 (block-wide reductions and barriers dominate on the small coarse
// grids, and they are cheaper with fewer warps).
static int coarse_threads(const Grid& g) {
    const long long t = ((g.size + 31) / 32) * 32;
    return (int)(t < 64 ? 64 : (t > kCoarseThreads ? kCoarseThreads : t));
}

// element contributions per element: 2^d (scalar) or 24 (beam)
__host__ __device__ inline int coarse_npe(const Grid& g) { return g.beam ? 24 : (g.d == 3 ? 8 : 4); }

template <typename T, Prob P>
__device__ void coarse_apply_A(const Grid& g, const T* w, T* elemC, T* out, const T* kappa, T lh, T node_scale) {
    // elemC: [nelem][npe];  out: A(w) scaled, full grid (boundary entries untouched)
    const int n = g.n;
    const int tid = threadIdx.x;
    if (P == Prob::BEAM3) {
        // lh = 1/h; 10n x n x n elements, 3 components per node
        const int ex = 10 * n, ne = ex * n * n;
        for (int e = tid; e < ne; e += blockDim.x) {
            const int x = e % ex, y = (e / ex) % n, z = e / (ex * n);
            T ue[24], r[24];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int node = ((z + (c >> 2)) * g.ny + y + ((c >> 1) & 1)) * g.nx + x + (c & 1);
#pragma unroll
                for (int i = 0; i < 3; ++i) ue[3 * c + i] = w[node * 3 + i];
            }
            elem_neohooke<T>(ue, lh, r);
#pragma unroll
            for (int k = 0; k < 24; ++k) elemC[e * 24 + k] = r[k];
        }
        __syncthreads();
        for (long long k = tid; k < g.size; k += blockDim.x) {
            const int i = (int)(k % 3);
            const int node = (int)(k / 3);
            const int X = node % g.nx, Y = (node / g.nx) % g.ny, Z = node / (g.nx * g.ny);
            T acc = T(0);
            for (int c = 0; c < 8; ++c) {
                const int xe = X - (c & 1), ye = Y - ((c >> 1) & 1), ze = Z - (c >> 2);
                if (xe < 0 || xe >= ex || ye < 0 || ye >= n || ze < 0 || ze >= n) continue;
                acc += elemC[((ze * n + ye) * ex + xe) * 24 + 3 * c + i];
            }
            out[k] = acc;
        }
    } else if (is_2d(P)) {
        const int ne = n * n;
        for (int e = tid; e < ne; e += blockDim.x) {
            const int ex = e % n, ey = e / n;
            const long long b = (long long)ey * g.sy + ex;
            T ue[4] = {w[b], w[b + 1], w[b + g.sy], w[b + g.sy + 1]};
            T r[4];
            if (P == Prob::MINSURF2)
                elem_minsurf2<T>(ue, lh, r);
            else
                elem_bratu2<T>(ue, lh, r);
#pragma unroll
            for (int c = 0; c < 4; ++c) elemC[e * 4 + c] = r[c];
        }
        __syncthreads();
        for (long long i = tid; i < g.size; i += blockDim.x) {
            const int x = (int)(i % g.sy), y = (int)(i / g.sy);
            T acc = T(0);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ex = x - 1 + a, ey = y - 1 + b;  // element with the node at local (1-a, 1-b)
                    if (ex >= 0 && ex < n && ey >= 0 && ey < n) acc += elemC[(ey * n + ex) * 4 + (1 - a) + 2 * (1 - b)];
                }
            out[i] = acc * node_scale;
        }
    } else {
        const int ne = n * n * n;
        for (int e = tid; e < ne; e += blockDim.x) {
            const int ex = e % n, ey = (e / n) % n, ez = e / (n * n);
            const long long b = (long long)ez * g.sz + (long long)ey * g.sy + ex;
            T ue[8] = {w[b],        w[b + 1],        w[b + g.sy],        w[b + g.sy + 1],
                       w[b + g.sz], w[b + g.sz + 1], w[b + g.sz + g.sy], w[b + g.sz + g.sy + 1]};
            T r[8];
            if (P == Prob::NDK3)
                elem_nd3<T, true>(ue, kappa[e], r);
            else
                elem_nd3<T, false>(ue, T(1), r);
#pragma unroll
            for (int c = 0; c < 8; ++c) elemC[e * 8 + c] = r[c];
        }
        __syncthreads();
        for (long long i = tid; i < g.size; i += blockDim.x) {
            const int x = (int)(i % g.sy);
            const int y = (int)((i / g.sy) % g.ny);
            const int z = (int)(i / g.sz);
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const int ex = x - 1 + a, ey = y - 1 + b, ez = z - 1 + c;
                        if (ex >= 0 && ex < n && ey >= 0 && ey < n && ez >= 0 && ez < n)
                            acc += elemC[((ez * n + ey) * n + ex) * 8 + (1 - a) + 2 * (1 - b) + 4 * (1 - c)];
                    }
            out[i] = acc * node_scale;
        }
    }
    __syncthreads();
}

// J(x)^T v on the coarse grid (3D diffusion problems), full grid out (boundary untouched)
template <typename T, Prob P>
__device__ void coarse_apply_vjp(const Grid& g, const T* x, const T* v, T* elemC, T* out, const T* kappa,
                                 T node_scale) {
    const int n = g.n;
    const int tid = threadIdx.x;
    const int ne = n * n * n;
    for (int e = tid; e < ne; e += blockDim.x) {
        const int ex = e % n, ey = (e / n) % n, ez = e / (n * n);
        const long long b = (long long)ez * g.sz + (long long)ey * g.sy + ex;
        const long long o[8] = {0, 1, g.sy, g.sy + 1, g.sz, g.sz + 1, g.sz + g.sy, g.sz + g.sy + 1};
        T ue[8], ve[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            ue[c] = x[b + o[c]];
            ve[c] = v[b + o[c]];
        }
        T r[8], dk;
        elem_vjp3<T>(ue, ve, P == Prob::NDK3 ? kappa[e] : T(1), r, dk);
#pragma unroll
        for (int c = 0; c < 8; ++c) elemC[e * 8 + c] = r[c];
    }
    __syncthreads();
    for (long long i = tid; i < g.size; i += blockDim.x) {
        const int xx = (int)(i % g.sy);
        const int yy = (int)((i / g.sy) % g.ny);
        const int zz = (int)(i / g.sz);
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ex = xx - 1 + a, ey = yy - 1 + bb, ez = zz - 1 + c;
                    if (ex >= 0 && ex < n && ey >= 0 && ey < n && ez >= 0 && ez < n)
                        acc += elemC[((ez * n + ey) * n + ex) * 8 + (1 - a) + 2 * (1 - bb) + 4 * (1 - c)];
                }
        out[i] = acc * node_scale;
    }
    __syncthreads();
}

__device__ __forceinline__ bool coarse_inner(const Grid& g, long long i) { return grid_unknown(g, i); }

// vsm: the Krylov basis V and the Hessenberg matrix H live in shared memory
// (after the work arrays) instead of the global scratch a.V / a.H
template <typename T, Prob P, bool ADJ>
__device__ void coarse_gmres_body(const CoarseArgs<T>& a, unsigned char* smem_raw, bool vsm) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const int ne = (int)g.elements();
    const int npe = coarse_npe(g);
    const int m = a.maxit;
    T* wv = reinterpret_cast<T*>(smem_raw);  // [N] work vector
    T* xw = wv + N;                          // [N] x + eps v
    T* Aw = xw + N;                          // [N] A(x + eps v)
    T* elemC = Aw + N;                       // [ne * npe]
    double* hcol = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(elemC + ne * npe) + 15) & ~uintptr_t(15));  // [m + 1]
    double* cs = hcol + (m + 1);             // [m]
    double* sn = cs + m;                     // [m]
    double* gv = sn + m;                     // [m + 1]
    double* red = gv + (m + 1);              // [32]
    __shared__ double s_scalar[4];
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    const int lane = tid & 31, wid = tid >> 5;
    T* V = a.V;       // (m + 1) x N
    double* H = a.H;  // (m + 1) x m, column-major: H[j * (m+1) + i]
    if (vsm) {
        H = red + 32;
        V = reinterpret_cast<T*>(H + (size_t)(m + 1) * m);
    }

    // ||b|| over interior; V_0 = b / ||b||
    double acc = 0.0;
    for (int i = tid; i < N; i += blockDim.x)
        if (coarse_inner(g, i)) acc += (double)a.b[i] * (double)a.b[i];
    double bn = block_sum(acc, red);
    if (tid == 0) s_scalar[0] = sqrt(bn);
    __syncthreads();
    const double beta = s_scalar[0];
    const double target = a.tol_abs ? a.tol : a.tol * beta;
    int k = 0;
    if (!(beta > 0.0) || beta <= target) {
        for (int i = tid; i < N; i += blockDim.x) a.s[i] = T(0);
        return;
    }
    for (int i = tid; i < N; i += blockDim.x) V[i] = coarse_inner(g, i) ? (T)((double)a.b[i] / beta) : T(0);
    if (tid == 0) {
        gv[0] = beta;
        for (int j = 1; j <= m; ++j) gv[j] = 0.0;
        s_flag = 0;
    }
    __syncthreads();
    const double xstat = *a.xstat;
    for (int j = 0; j < m; ++j) {
        const T* vj = V + (long long)j * N;
        // ||v_j|| (unit up to rounding) and the FD step
        T vacc = T(0);
        for (int i = tid; i < N; i += blockDim.x)
            if (coarse_inner(g, i)) vacc += vj[i] * vj[i];
        double vn2 = block_sum(vacc, red);
        if (tid == 0) {
            double e = eps_formula(a.eps_mode, a.n_unknowns, xstat, sqrt(vn2));
            s_scalar[1] = e;
            s_scalar[2] = e > 0.0 ? 1.0 / e : 0.0;
        }
        __syncthreads();
        if (ADJ) {
            // adjoint operator: J(x_0)^T v_j, exact, element by element
            for (int i = tid; i < N; i += blockDim.x) xw[i] = coarse_inner(g, i) ? vj[i] : T(0);
            __syncthreads();
            coarse_apply_vjp<T, P>(g, a.x, xw, elemC, Aw, a.kappa, a.node_scale);
            for (int i = tid; i < N; i += blockDim.x) wv[i] = coarse_inner(g, i) ? Aw[i] : T(0);
        } else {
            const T eps = (T)s_scalar[1], inv_eps = (T)s_scalar[2];
            for (int i = tid; i < N; i += blockDim.x) xw[i] = a.x[i] + (coarse_inner(g, i) ? eps * vj[i] : T(0));
            __syncthreads();
            coarse_apply_A<T, P>(g, xw, elemC, Aw, a.kappa, a.lh, a.node_scale);
            for (int i = tid; i < N; i += blockDim.x) wv[i] = coarse_inner(g, i) ? (Aw[i] - a.Ax[i]) * inv_eps : T(0);
        }
        __syncthreads();
        // classical Gram-Schmidt, twice; h accumulated in hcol
        for (int i = tid; i <= j; i += blockDim.x) hcol[i] = 0.0;
        __syncthreads();
        // (dots and updates in the basis precision T: in an FP32 preconditioner the
        // single CTA would otherwise spend its iterations on this SM's FP64 pipe,
        // 1/74 of the FP32 rate; the Hessenberg entries are kept in FP64)
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = wid; q <= j; q += nwarps) {
                const T* vq = V + (long long)q * N;
                T d = T(0);
                for (int i = lane; i < N; i += 32) d += wv[i] * vq[i];
                d = warp_sum(d);
                if (lane == 0) {
                    hcol[q] += (double)d;
                    H[(long long)j * (m + 1) + q] = (double)d;
                }
            }
            __syncthreads();
            for (int i = tid; i < N; i += blockDim.x) {
                T w = wv[i];
                for (int q = 0; q <= j; ++q) w -= (T)H[(long long)j * (m + 1) + q] * V[(long long)q * N + i];
                wv[i] = w;
            }
            __syncthreads();
        }
        T accT = T(0);
        for (int i = tid; i < N; i += blockDim.x) accT += wv[i] * wv[i];
        double wn2 = block_sum(accT, red);
        if (tid == 0) {
            const double hn = sqrt(wn2);
            hcol[j + 1] = hn;
            // Givens: apply previous rotations to column j, then the new one
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = t;
            }
            double aa = hcol[j], bb = hcol[j + 1];
            double c = 1.0, s = 0.0;
            if (bb != 0.0) {
                double r = hypot(aa, bb);
                c = aa / r;
                s = bb / r;
            }
            cs[j] = c;
            sn[j] = s;
            hcol[j] = c * aa + s * bb;
            hcol[j + 1] = 0.0;
            gv[j + 1] = -s * gv[j];
            gv[j] = c * gv[j];
            for (int i = 0; i <= j; ++i) H[(long long)j * (m + 1) + i] = hcol[i];
            const double res = fabs(gv[j + 1]);
            s_flag = (res <= target || !(hn > 0.0) || !isfinite(res)) ? 1 : 0;
            s_scalar[0] = hn;
        }
        __syncthreads();
        k = j + 1;
        if (s_flag) break;
        const T hinv = (T)(1.0 / s_scalar[0]);
        T* vn = V + (long long)(j + 1) * N;
        for (int i = tid; i < N; i += blockDim.x) vn[i] = wv[i] * hinv;
        __syncthreads();
    }
    // back-substitution (thread 0), y into gv
    if (tid == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double t = gv[i];
            for (int q = i + 1; q < k; ++q) t -= H[(long long)q * (m + 1) + i] * gv[q];
            gv[i] = t / H[(long long)i * (m + 1) + i];
        }
        if (a.iters) *a.iters += k;
    }
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) {
        T sv = T(0);
        for (int q = 0; q < k; ++q) sv += (T)gv[q] * V[(long long)q * N + i];
        a.s[i] = coarse_inner(g, i) ? sv : T(0);
    }
}

// ---------------------------------------------------------------------------
// The paper's coarse solver (Sec. 2 "The coarse level solver", Alg. 1, l = 0):
// CG preconditioned by L-BFGS, stopped on negative curvature, and re-run on the
// shifted operator A_s = A - lambda_c+ I (lambda_c+ <= 0) with
// lambda_c+ <- gamma min(lambda_c, lambda_c+) while the Rayleigh quotient
// lambda_c = p.A_s p / p.p of the direction of negative curvature is < 0.
// The secant pairs (s_i, y_i) = (alpha_i p_i, alpha_i A p_i) of the very first
// call are collected; m of the k steps, those of iterations floor(j k / m),
// are kept (uniform sampling) and define the preconditioner for the rest of
// the solve.  Each shifted call restarts CG from the returned s_0.  At most
// 30 shifted calls.  All of it runs in one CTA.
// ---------------------------------------------------------------------------
constexpr int kMaxShiftCalls = 30;

// block-wide interior dot product, result in every thread
template <typename T>
__device__ double cg_dot(const Grid& g, const T* a, const T* b, int N, double* red, double* bc) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        if (coarse_inner(g, i)) acc += (double)a[i] * (double)b[i];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) *bc = t;
    __syncthreads();
    const double r = *bc;
    __syncthreads();
    return r;
}

// q = A_s p = (A(x_0 + eps p) - A(x_0)) / eps - shift p on interior nodes, 0 on the boundary
template <typename T, Prob P>
__device__ void cg_apply(const CoarseArgs<T>& a, const T* p, T* q, T* xw, T* Aw, T* elemC, double shift,
                         double xstat, double* red, double* bc) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const double pn = sqrt(cg_dot(g, p, p, N, red, bc));
    const double e = eps_formula(a.eps_mode, a.n_unknowns, xstat, pn);
    if (!(e > 0.0) || !isfinite(e)) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) q[i] = T(0);
        __syncthreads();
        return;
    }
    const T eps = (T)e, inv = (T)(1.0 / e), sh = (T)shift;
    for (int i = threadIdx.x; i < N; i += blockDim.x) xw[i] = a.x[i] + (coarse_inner(g, i) ? eps * p[i] : T(0));
    __syncthreads();
    coarse_apply_A<T, P>(g, xw, elemC, Aw, a.kappa, a.lh, a.node_scale);
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        q[i] = coarse_inner(g, i) ? (Aw[i] - a.Ax[i]) * inv - sh * p[i] : T(0);
    __syncthreads();
}

// z = H r with the compact L-BFGS form (k kept pairs; k = 0: z = r)
template <typename T>
__device__ void cg_precond(const CoarseArgs<T>& a, const T* r, T* z, int k, double* dots, double* coef) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    if (k <= 0) {
        for (int i = tid; i < N; i += blockDim.x) z[i] = r[i];
        __syncthreads();
        return;
    }
    const LbfgsState* lb = a.lb;
    for (int q = wid; q < 2 * k; q += nwarps) {
        const T* v = (q < k) ? a.S + (long long)q * N : a.Y + (long long)(q - k) * N;
        double d = 0.0;
        for (int i = lane; i < N; i += 32) d += (double)v[i] * (double)r[i];
        d = warp_sum(d);
        if (lane == 0) dots[q] = d;
    }
    __syncthreads();
    if (tid == 0) {
        const double gam = lb->gamma;
        double t[kMaxLbfgsPairs], v[kMaxLbfgsPairs];
        // t = R^-1 (S^T r)
        for (int i = k - 1; i >= 0; --i) {
            double acc = dots[i];
            for (int j = i + 1; j < k; ++j) acc -= lb->R[i * kMaxLbfgsPairs + j] * t[j];
            t[i] = acc / lb->R[i * kMaxLbfgsPairs + i];
        }
        // v = (D + gamma Y^T Y) t - gamma Y^T r
        for (int i = 0; i < k; ++i) {
            double acc = lb->R[i * kMaxLbfgsPairs + i] * t[i];
            for (int j = 0; j < k; ++j) acc += gam * lb->YtY[i * kMaxLbfgsPairs + j] * t[j];
            v[i] = acc - gam * dots[k + i];
        }
        // top = R^-T v ; coefficients of S (top) and of Y (-gamma t)
        for (int i = 0; i < k; ++i) {
            double acc = v[i];
            for (int j = 0; j < i; ++j) acc -= lb->R[j * kMaxLbfgsPairs + i] * coef[j];
            coef[i] = acc / lb->R[i * kMaxLbfgsPairs + i];
        }
        for (int i = 0; i < k; ++i) coef[k + i] = -gam * t[i];
        coef[2 * k] = gam;
    }
    __syncthreads();
    const double gam = coef[2 * k];
    for (int i = tid; i < N; i += blockDim.x) {
        double acc = gam * (double)r[i];
        for (int j = 0; j < k; ++j)
            acc += coef[j] * (double)a.S[(long long)j * N + i] + coef[k + j] * (double)a.Y[(long long)j * N + i];
        z[i] = coarse_inner(g, i) ? (T)acc : T(0);
    }
    __syncthreads();
}

struct CgOut {
    double lam_c;  // Rayleigh quotient at negative curvature, else 0
    int its;
    int fd;        // FD actions (level-0 gradient evaluations)
    int negcurv;
};

// CG(s_0, x_0, F(x_0), r_0, lambda_c+) of Alg. 1 on the vectors in shared memory
template <typename T, Prob P>
__device__ CgOut coarse_cg_run(const CoarseArgs<T>& a, T* x, T* r, T* z, T* pv, T* q, T* xw, T* Aw, T* elemC,
                               double shift, bool warm, int kpre, bool collect, double xstat, double target,
                               double* red, double* bc, double* dots, double* coef) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const int tid = threadIdx.x;
    CgOut o = {0.0, 0, 0, 0};
    if (warm) {
        cg_apply<T, P>(a, x, q, xw, Aw, elemC, shift, xstat, red, bc);
        o.fd++;
        for (int i = tid; i < N; i += blockDim.x) r[i] = coarse_inner(g, i) ? a.b[i] - q[i] : T(0);
    } else {
        for (int i = tid; i < N; i += blockDim.x) r[i] = coarse_inner(g, i) ? a.b[i] : T(0);
    }
    __syncthreads();
    double res = sqrt(cg_dot(g, r, r, N, red, bc));
    if (!(res > 0.0) || res <= target || !isfinite(res)) return o;
    cg_precond<T>(a, r, z, kpre, dots, coef);
    double rz = cg_dot(g, r, z, N, red, bc);
    for (int i = tid; i < N; i += blockDim.x) pv[i] = z[i];
    __syncthreads();
    for (int it = 1; it <= a.maxit; ++it) {
        cg_apply<T, P>(a, pv, q, xw, Aw, elemC, shift, xstat, red, bc);
        o.fd++;
        o.its = it;
        const double pq = cg_dot(g, pv, q, N, red, bc);
        if (!isfinite(pq)) return o;
        if (pq <= 0.0) {
            const double pp = cg_dot(g, pv, pv, N, red, bc);
            o.lam_c = pp > 0.0 ? pq / pp : 0.0;
            o.negcurv = 1;
            return o;
        }
        const double alpha = rz / pq;
        const T al = (T)alpha;
        for (int i = tid; i < N; i += blockDim.x) {
            if (collect) {
                a.S_all[(long long)(it - 1) * N + i] = al * pv[i];
                a.Y_all[(long long)(it - 1) * N + i] = al * q[i];
            }
            x[i] += al * pv[i];
            r[i] -= al * q[i];
        }
        if (collect && tid == 0) a.lb->collected = it;
        __syncthreads();
        res = sqrt(cg_dot(g, r, r, N, red, bc));
        if (res <= target || !isfinite(res)) return o;
        cg_precond<T>(a, r, z, kpre, dots, coef);
        const double rz_new = cg_dot(g, r, z, N, red, bc);
        const T beta = (T)(rz_new / rz);
        rz = rz_new;
        for (int i = tid; i < N; i += blockDim.x) pv[i] = z[i] + beta * pv[i];
        __syncthreads();
    }
    return o;
}

// keep m of the collected pairs (uniform sampling) and set up the compact form
template <typename T>
__device__ void lbfgs_build(const CoarseArgs<T>& a, double* red, double* bc) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    LbfgsState* lb = a.lb;
    const int kall = lb->collected;
    const int m = min(a.m_pairs, kMaxLbfgsPairs);
    const int k = min(kall, m);
    for (int j = 0; j < k; ++j) {
        const long long src = (kall > m) ? ((long long)j * kall) / m : j;
        for (int i = tid; i < N; i += blockDim.x) {
            a.S[(long long)j * N + i] = a.S_all[src * N + i];
            a.Y[(long long)j * N + i] = a.Y_all[src * N + i];
        }
    }
    __syncthreads();
    // R_ij = s_i.y_j (i <= j), YtY_ij = y_i.y_j
    for (int q = wid; q < 2 * k * k; q += nwarps) {
        const int which = q / (k * k), ij = q % (k * k), i = ij / k, j = ij % k;
        const T* u = (which == 0) ? a.S + (long long)i * N : a.Y + (long long)i * N;
        const T* v = a.Y + (long long)j * N;
        double d = 0.0;
        for (int t = lane; t < N; t += 32) d += (double)u[t] * (double)v[t];
        d = warp_sum(d);
        if (lane == 0) {
            if (which == 0)
                lb->R[i * kMaxLbfgsPairs + j] = (i <= j) ? d : 0.0;
            else
                lb->YtY[i * kMaxLbfgsPairs + j] = d;
        }
    }
    __syncthreads();
    if (tid == 0) {
        bool ok = k > 0;
        for (int i = 0; i < k; ++i) ok = ok && lb->R[i * kMaxLbfgsPairs + i] > 0.0;
        const double yy = k > 0 ? lb->YtY[(k - 1) * kMaxLbfgsPairs + (k - 1)] : 0.0;
        lb->gamma = (ok && yy > 0.0) ? lb->R[(k - 1) * kMaxLbfgsPairs + (k - 1)] / yy : 1.0;
        lb->count = (ok && yy > 0.0) ? k : 0;
    }
    __syncthreads();
}

template <typename T, Prob P>
__global__ void __launch_bounds__(kCoarseThreads) coarse_cgqn_kernel(CoarseArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Grid g = a.g;
    const int N = (int)g.size;
    const int ne = (int)g.elements();
    const int npe = coarse_npe(g);
    T* x = reinterpret_cast<T*>(smem_raw);
    T* r = x + N;
    T* z = r + N;
    T* pv = z + N;
    T* q = pv + N;
    T* xw = q + N;
    T* Aw = xw + N;
    T* elemC = Aw + N;
    double* dd = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(elemC + ne * npe) + 15) & ~uintptr_t(15));
    double* dots = dd;                        // [2 kMax]
    double* coef = dots + 2 * kMaxLbfgsPairs;  // [2 kMax + 1]
    double* red = coef + 2 * kMaxLbfgsPairs + 2;  // [32]
    __shared__ double bc;
    __shared__ int s_count;
    const int tid = threadIdx.x;
    const double xstat = *a.xstat;
    const double bn = sqrt(cg_dot(g, a.b, a.b, N, red, &bc));
    const double target = a.tol_abs ? a.tol : a.tol * bn;
    for (int i = tid; i < N; i += blockDim.x) x[i] = T(0);
    if (tid == 0) s_count = a.lb->count;
    __syncthreads();
    const bool collect = s_count < 0;
    long long fd = 0;
    int negc = 0;
    double shift = 0.0;
    CgOut o = coarse_cg_run<T, P>(a, x, r, z, pv, q, xw, Aw, elemC, shift, false, collect ? 0 : s_count, collect,
                                  xstat, target, red, &bc, dots, coef);
    fd += o.fd;
    negc += o.negcurv;
    if (collect) {
        lbfgs_build<T>(a, red, &bc);
        if (tid == 0) s_count = a.lb->count;
        __syncthreads();
    }
    int nshift = 0;
    while (o.lam_c < 0.0 && nshift < kMaxShiftCalls) {
        shift = a.shift_gamma * fmin(o.lam_c, shift);
        ++nshift;
        o = coarse_cg_run<T, P>(a, x, r, z, pv, q, xw, Aw, elemC, shift, true, s_count, false, xstat, target, red,
                                &bc, dots, coef);
        fd += o.fd;
        negc += o.negcurv;
    }
    for (int i = tid; i < N; i += blockDim.x) a.s[i] = coarse_inner(g, i) ? x[i] : T(0);
    if (tid == 0) {
        if (a.iters) *a.iters += fd;
        a.lb->shifts += nshift;
        a.lb->negcurv += negc;
    }
}

size_t coarse_cgqn_smem_bytes(const Grid& g, size_t esz) {
    const int ne = (int)g.elements();
    const int npe = coarse_npe(g);
    size_t b = esz * (7 * (size_t)g.size + (size_t)ne * npe);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * (4 * kMaxLbfgsPairs + 2 + 32);
    return b;
}

template <typename T, Prob P, bool ADJ>
__global__ void __launch_bounds__(kCoarseThreads) coarse_gmres_kernel(CoarseArgs<T> a, int vsm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    coarse_gmres_body<T, P, ADJ>(a, smem_raw, vsm != 0);
}

// one CTA per instance of a batch (all instances share the coarse grid size)
template <typename T, Prob P, bool ADJ>
__global__ void __launch_bounds__(kCoarseThreads) coarse_gmres_batched_kernel(const CoarseArgs<T>* args, int vsm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CoarseArgs<T> a = args[blockIdx.x];
    coarse_gmres_body<T, P, ADJ>(a, smem_raw, vsm != 0);
}

// Shared memory of the GMRES kernel: work arrays, plus V and H when vsm.
template <typename T>
size_t coarse_smem_bytes(const Grid& g, int maxit, bool vsm) {
    const int ne = (int)g.elements();
    const int npe = coarse_npe(g);
    size_t b = sizeof(T) * (3 * (size_t)g.size + (size_t)ne * npe);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * (4 * (size_t)maxit + 2 + 32);
    if (vsm) b += sizeof(double) * (size_t)(maxit + 1) * maxit + sizeof(T) * (size_t)(maxit + 1) * g.size;
    return b;
}

// V and H go to shared memory when everything fits in kCoarseVsmBytes (the
// basis is then read at shared-memory rather than L2 latency in the
// orthogonalisation, the critical path of this one-CTA solver)
constexpr size_t kCoarseVsmBytes = 160 * 1024;
template <typename T>
static bool coarse_vsm(const Grid& g, int maxit) {
    return coarse_smem_bytes<T>(g, maxit, true) <= kCoarseVsmBytes;
}

template <typename T>
static jfnk_status launch_coarse_cgqn(Prob prob, const CoarseArgs<T>& a, cudaStream_t st) {
    if (a.adjoint) {
        set_error("the CG-QN coarse solver is implemented for the forward operator");
        return JFNK_ERR_NOT_IMPLEMENTED;
    }
    if (!a.lb || !a.S_all || !a.Y_all || !a.S || !a.Y || a.m_pairs < 1 || a.m_pairs > kMaxLbfgsPairs) {
        set_error("CG-QN coarse solver: workspace not laid out for it, or 1 <= pairs <= %d violated", kMaxLbfgsPairs);
        return JFNK_ERR_WORKSPACE;
    }
    const size_t smem = coarse_cgqn_smem_bytes(a.g, sizeof(T));
    if (smem > 200 * 1024) {
        set_error("coarse solver shared memory %zu too large", smem);
        return JFNK_ERR_INVALID_ARG;
    }
#define JFNK_CGQN_LAUNCH(PP)                                                                         \
    do {                                                                                             \
        JFNK_CUDA_TRY(cudaFuncSetAttribute(coarse_cgqn_kernel<T, PP>,                                 \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        coarse_cgqn_kernel<T, PP><<<1, coarse_threads(a.g), smem, st>>>(a);                                \
    } while (0)
    switch (prob) {
        case Prob::BRATU2: JFNK_CGQN_LAUNCH(Prob::BRATU2); break;
        case Prob::MINSURF2: JFNK_CGQN_LAUNCH(Prob::MINSURF2); break;
        case Prob::BEAM3: JFNK_CGQN_LAUNCH(Prob::BEAM3); break;
        case Prob::ND3: JFNK_CGQN_LAUNCH(Prob::ND3); break;
        case Prob::NDK3: JFNK_CGQN_LAUNCH(Prob::NDK3); break;
    }
#undef JFNK_CGQN_LAUNCH
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T>
jfnk_status launch_coarse(Prob prob, const CoarseArgs<T>& a, cudaStream_t st) {
    if (a.g.size > JFNK_COARSE_MAX_NODES || a.maxit > JFNK_COARSE_MAX_IT || a.maxit < 1) {
        set_error("coarse grid too large for the single-CTA solver (%lld nodes, maxit %d)", a.g.size, a.maxit);
        return JFNK_ERR_INVALID_ARG;
    }
    if (a.method == 1) return launch_coarse_cgqn<T>(prob, a, st);
    const bool vsm = coarse_vsm<T>(a.g, a.maxit);
    const size_t smem = coarse_smem_bytes<T>(a.g, a.maxit, vsm);
    if (smem > 200 * 1024) {
        set_error("coarse solver shared memory %zu too large", smem);
        return JFNK_ERR_INVALID_ARG;
    }
    if (a.adjoint && is_2d(prob)) {
        set_error("the adjoint coarse solve is implemented for the 3D diffusion problems");
        return JFNK_ERR_NOT_IMPLEMENTED;
    }
#define JFNK_COARSE_LAUNCH(PP, ADJ)                                                                  \
    do {                                                                                             \
        JFNK_CUDA_TRY(cudaFuncSetAttribute(coarse_gmres_kernel<T, PP, ADJ>,                           \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        coarse_gmres_kernel<T, PP, ADJ><<<1, coarse_threads(a.g), smem, st>>>(a, vsm ? 1 : 0);             \
    } while (0)
    switch (prob) {
        case Prob::BRATU2: JFNK_COARSE_LAUNCH(Prob::BRATU2, false); break;
        case Prob::MINSURF2: JFNK_COARSE_LAUNCH(Prob::MINSURF2, false); break;
        case Prob::BEAM3:
            if (a.adjoint) {
                set_error("no adjoint for the beam");
                return JFNK_ERR_NOT_IMPLEMENTED;
            }
            JFNK_COARSE_LAUNCH(Prob::BEAM3, false);
            break;
        case Prob::ND3:
            if (a.adjoint) JFNK_COARSE_LAUNCH(Prob::ND3, true);
            else JFNK_COARSE_LAUNCH(Prob::ND3, false);
            break;
        case Prob::NDK3:
            if (a.adjoint) JFNK_COARSE_LAUNCH(Prob::NDK3, true);
            else JFNK_COARSE_LAUNCH(Prob::NDK3, false);
            break;
    }
#undef JFNK_COARSE_LAUNCH
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template jfnk_status launch_coarse<float>(Prob, const CoarseArgs<float>&, cudaStream_t);
template jfnk_status launch_coarse<double>(Prob, const CoarseArgs<double>&, cudaStream_t);
template <typename T>
jfnk_status launch_coarse_batched(const CoarseArgs<T>& a0, const CoarseArgs<T>* dev_args, int count, cudaStream_t st) {
    if (count <= 0) return JFNK_OK;
    if (a0.g.size > JFNK_COARSE_MAX_NODES || a0.maxit > JFNK_COARSE_MAX_IT || a0.maxit < 1 || a0.g.d != 2) {
        set_error("batched coarse solve: 2D coarse grids within the single-CTA limits only");
        return JFNK_ERR_INVALID_ARG;
    }
    const bool vsm = coarse_vsm<T>(a0.g, a0.maxit);
    const size_t smem = coarse_smem_bytes<T>(a0.g, a0.maxit, vsm);
    JFNK_CUDA_TRY(cudaFuncSetAttribute(coarse_gmres_batched_kernel<T, Prob::BRATU2, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    coarse_gmres_batched_kernel<T, Prob::BRATU2, false><<<count, coarse_threads(a0.g), smem, st>>>(dev_args,
                                                                                                   vsm ? 1 : 0);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status launch_coarse_batched<float>(const CoarseArgs<float>&, const CoarseArgs<float>*, int, cudaStream_t);
template jfnk_status launch_coarse_batched<double>(const CoarseArgs<double>&, const CoarseArgs<double>*, int, cudaStream_t);

}  // namespace jfnk
