// Coarse-level solve of Algorithm 1 (l = 0): a matrix-free Krylov method in
// place of a direct solver (Sec. 2, "The coarse level solver").  The configured
// workloads use unrestarted GMRES with x0 = 0; it stops when the Givens
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

template <typename T, Prob P>
__device__ void coarse_apply_A(const Grid& g, const T* w, T* elemC, T* out, const T* kappa, T lh, T node_scale) {
    // elemC: [nelem][2^d];  out: A(w) scaled, full grid (boundary entries untouched)
    const int n = g.n;
    const int tid = threadIdx.x;
    if (P == Prob::BRATU2) {
        const int ne = n * n;
        for (int e = tid; e < ne; e += blockDim.x) {
            const int ex = e % n, ey = e / n;
            const long long b = (long long)ey * g.sy + ex;
            T ue[4] = {w[b], w[b + 1], w[b + g.sy], w[b + g.sy + 1]};
            T r[4];
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

__device__ __forceinline__ bool coarse_inner(const Grid& g, long long i) {
    const int x = (int)(i % g.sy);
    const int y = (int)((i / g.sy) % g.ny);
    bool in = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1;
    if (g.d == 3) {
        const int z = (int)(i / g.sz);
        in = in && z > 0 && z < g.nz - 1;
    }
    return in;
}

template <typename T, Prob P, bool ADJ>
__device__ void coarse_gmres_body(const CoarseArgs<T>& a, unsigned char* smem_raw) {
    const Grid g = a.g;
    const int N = (int)g.size;
    const int ne = (g.d == 3) ? g.n * g.n * g.n : g.n * g.n;
    const int npe = (g.d == 3) ? 8 : 4;
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
    T* V = a.V;       // (m + 1) x N, global scratch
    double* H = a.H;  // (m + 1) x m, column-major: H[j * (m+1) + i]

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
        acc = 0.0;
        for (int i = tid; i < N; i += blockDim.x)
            if (coarse_inner(g, i)) acc += (double)vj[i] * (double)vj[i];
        double vn2 = block_sum(acc, red);
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
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = wid; q <= j; q += nwarps) {
                const T* vq = V + (long long)q * N;
                double d = 0.0;
                for (int i = lane; i < N; i += 32) d += (double)wv[i] * (double)vq[i];
                d = warp_sum(d);
                if (lane == 0) {
                    hcol[q] += d;
                    H[(long long)j * (m + 1) + q] = d;
                }
            }
            __syncthreads();
            for (int i = tid; i < N; i += blockDim.x) {
                double w = (double)wv[i];
                for (int q = 0; q <= j; ++q) w -= H[(long long)j * (m + 1) + q] * (double)V[(long long)q * N + i];
                wv[i] = (T)w;
            }
            __syncthreads();
        }
        acc = 0.0;
        for (int i = tid; i < N; i += blockDim.x) acc += (double)wv[i] * (double)wv[i];
        double wn2 = block_sum(acc, red);
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
        const double hn = s_scalar[0];
        T* vn = V + (long long)(j + 1) * N;
        for (int i = tid; i < N; i += blockDim.x) vn[i] = (T)((double)wv[i] / hn);
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
        double sv = 0.0;
        for (int q = 0; q < k; ++q) sv += gv[q] * (double)V[(long long)q * N + i];
        a.s[i] = coarse_inner(g, i) ? (T)sv : T(0);
    }
}

template <typename T, Prob P, bool ADJ>
__global__ void __launch_bounds__(kCoarseThreads) coarse_gmres_kernel(CoarseArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    coarse_gmres_body<T, P, ADJ>(a, smem_raw);
}

// one CTA per instance of a batch (all instances share the coarse grid size)
template <typename T, Prob P, bool ADJ>
__global__ void __launch_bounds__(kCoarseThreads) coarse_gmres_batched_kernel(const CoarseArgs<T>* args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CoarseArgs<T> a = args[blockIdx.x];
    coarse_gmres_body<T, P, ADJ>(a, smem_raw);
}

template <typename T>
size_t coarse_smem_bytes(const Grid& g, int maxit) {
    const int ne = (g.d == 3) ? g.n * g.n * g.n : g.n * g.n;
    const int npe = (g.d == 3) ? 8 : 4;
    size_t b = sizeof(T) * (3 * (size_t)g.size + (size_t)ne * npe);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * (4 * (size_t)maxit + 2 + 32);
    return b;
}

template <typename T>
jfnk_status launch_coarse(Prob prob, const CoarseArgs<T>& a, cudaStream_t st) {
    if (a.g.size > JFNK_COARSE_MAX_NODES || a.maxit > JFNK_COARSE_MAX_IT || a.maxit < 1) {
        set_error("coarse grid too large for the single-CTA solver (%lld nodes, maxit %d)", a.g.size, a.maxit);
        return JFNK_ERR_INVALID_ARG;
    }
    const size_t smem = coarse_smem_bytes<T>(a.g, a.maxit);
    if (smem > 200 * 1024) {
        set_error("coarse solver shared memory %zu too large", smem);
        return JFNK_ERR_INVALID_ARG;
    }
    if (a.adjoint && prob == Prob::BRATU2) {
        set_error("the adjoint coarse solve is implemented for the 3D diffusion problems");
        return JFNK_ERR_NOT_IMPLEMENTED;
    }
#define JFNK_COARSE_LAUNCH(PP, ADJ)                                                                  \
    do {                                                                                             \
        JFNK_CUDA_TRY(cudaFuncSetAttribute(coarse_gmres_kernel<T, PP, ADJ>,                           \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        coarse_gmres_kernel<T, PP, ADJ><<<1, kCoarseThreads, smem, st>>>(a);                          \
    } while (0)
    switch (prob) {
        case Prob::BRATU2: JFNK_COARSE_LAUNCH(Prob::BRATU2, false); break;
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
    const size_t smem = coarse_smem_bytes<T>(a0.g, a0.maxit);
    JFNK_CUDA_TRY(cudaFuncSetAttribute(coarse_gmres_batched_kernel<T, Prob::BRATU2, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    coarse_gmres_batched_kernel<T, Prob::BRATU2, false><<<count, kCoarseThreads, smem, st>>>(dev_args);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status launch_coarse_batched<float>(const CoarseArgs<float>&, const CoarseArgs<float>*, int, cudaStream_t);
template jfnk_status launch_coarse_batched<double>(const CoarseArgs<double>&, const CoarseArgs<double>*, int, cudaStream_t);

}  // namespace jfnk
