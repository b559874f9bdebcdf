// Element-parallel 3D element-residual kernels.
//
// Phase 1 (elements): one thread per element gathers its 8 nodal values of
// w = x + eps v (boundary entries of v ignored), evaluates the element
// residual (or its vector-Jacobian product) and stores the 8 nodal
// contributions in a scratch array C[corner][element].  No shared memory and
// no barrier: every element of the level is independent, so all SMs stay busy
// whatever the grid size, and no element is evaluated twice.
// Phase 2 (nodes): one thread per node sums the contributions of its 8
// elements in a fixed order, applies the node factor and the fused epilogue of
// the mode, and the last block completes the norm reduction (deterministic).
//
// Each F_i is the same sum of element integrals as in the tiled kernels; the
// price is 2 x 8 scratch words per element of extra traffic, which the FP64
// kernels (bound by the FP64 pipe by two orders of magnitude) do not notice
// and which stays in L2 on the small levels.
#include <algorithm>

#include "element.cuh"
#include "reduce.cuh"
#include "stencil.cuh"
#include "stencil_body.cuh"
#include "stencil_ep.cuh"

namespace jfnk {

constexpr int kEpElemThreads = 128;
constexpr int kEpNodeThreads = 256;

template <typename T, Prob P, Mode M, bool ADJ>
__global__ void __launch_bounds__(kEpElemThreads) ep3d_elem_kernel(const StencilArgs<T> a) {
    const Grid g = a.g;
    const int n = g.n;
    const long long ne = (long long)n * n * n;
    T* C = a.face;
    T eps = T(0);
    if (!ADJ && M != Mode::F) eps = eps_of<T>(a.eps);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % n);
        const long long q = e / n;
        const int y = (int)(q % n), z = (int)(q / n);
        const long long base = (long long)z * g.sz + (long long)y * g.sy + x;
        T ue[8], ve[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
            const long long idx = base + dx + dy * g.sy + dz * g.sz;
            const int X = x + dx, Y = y + dy, Z = z + dz;
            const bool bnd = X == 0 || X == n || Y == 0 || Y == n || Z == 0 || Z == n;
            T uv = a.u[idx];
            if (ADJ) {
                ve[c] = bnd ? T(0) : a.v[idx];
            } else if (M != Mode::F) {
                if (!bnd) uv += eps * a.v[idx];
            }
            ue[c] = uv;
        }
        T r[8];
        if (ADJ) {
            T dk;
            elem_vjp3<T>(ue, ve, P == Prob::NDK3 ? a.kappa[e] : T(1), r, dk);
            if (a.dkout) a.dkout[e] = dk * a.dk_scale;
        } else if (P == Prob::NDK3) {
            elem_nd3<T, true>(ue, a.kappa[e], r);
        } else {
            elem_nd3<T, false>(ue, T(1), r);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) C[c * ne + e] = r[c];
    }
}

template <typename T, Mode M, bool ADJ>
__global__ void __launch_bounds__(kEpNodeThreads) ep3d_node_kernel(const StencilArgs<T> a) {
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int n = g.n, NP = n + 1;
    const long long ne = (long long)n * n * n;
    const long long nn = (long long)NP * NP * NP;
    const long long sy = n, sz = (long long)n * n;  // element strides
    const T* C = a.face;
    T inv_eps = T(0);
    if (!ADJ && M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
         i += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(i % NP);
        const long long q = i / NP;
        const int Y = (int)(q % NP), Z = (int)(q / NP);
        const long long idx = (long long)Z * g.sz + (long long)Y * g.sy + X;
        const bool inner = X > 0 && X < n && Y > 0 && Y < n && Z > 0 && Z < n;
        T val = T(0);
        if (inner) {
            // element with corner c = dx + 2 dy + 4 dz at this node: (X-dx, Y-dy, Z-dz)
            const long long e0 = (long long)Z * sz + (long long)Y * sy + X;
            const T c0 = C[0 * ne + e0], c1 = C[1 * ne + e0 - 1];
            const T c2 = C[2 * ne + e0 - sy], c3 = C[3 * ne + e0 - sy - 1];
            const T c4 = C[4 * ne + e0 - sz], c5 = C[5 * ne + e0 - sz - 1];
            const T c6 = C[6 * ne + e0 - sz - sy], c7 = C[7 * ne + e0 - sz - sy - 1];
            val = (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7))) * a.node_scale;
        }
        if (ADJ)
            epilogue_adj<T, M>(a, idx, inner, val, ck, red);
        else
            epilogue<T, M>(a, idx, inner, val, inv_eps, ck, red);
    }
    stencil_reduce(a, red, red_sm);
}

template <typename T, Prob P, Mode M, bool ADJ>
static jfnk_status launch_ep3d_pm(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    const long long ne = (long long)g.n * g.n * g.n;
    const long long nn = (long long)(g.n + 1) * (g.n + 1) * (g.n + 1);
    if (ep3d_scratch_count(g) > a.face_cap) {
        set_error("element scratch too small (%lld < %lld)", a.face_cap, ep3d_scratch_count(g));
        return JFNK_ERR_WORKSPACE;
    }
    const long long eb = std::min<long long>((ne + kEpElemThreads - 1) / kEpElemThreads, 1LL << 30);
    ep3d_elem_kernel<T, P, M, ADJ><<<(unsigned)eb, kEpElemThreads, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    // the reduction scratch holds 2 kMaxRedBlocks partials: grid-stride beyond
    const long long nb = std::min<long long>((nn + kEpNodeThreads - 1) / kEpNodeThreads, 2LL * kMaxRedBlocks);
    ep3d_node_kernel<T, M, ADJ><<<(unsigned)nb, kEpNodeThreads, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, Prob P, bool ADJ>
static jfnk_status launch_ep3d_p(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::F:
            if constexpr (!ADJ) return launch_ep3d_pm<T, P, Mode::F, false>(a, st);
            break;
        case Mode::JV: return launch_ep3d_pm<T, P, Mode::JV, ADJ>(a, st);
        case Mode::BMJ: return launch_ep3d_pm<T, P, Mode::BMJ, ADJ>(a, st);
        case Mode::CHEB0: return launch_ep3d_pm<T, P, Mode::CHEB0, ADJ>(a, st);
        case Mode::CHEB: return launch_ep3d_pm<T, P, Mode::CHEB, ADJ>(a, st);
        case Mode::CHEBLAST: return launch_ep3d_pm<T, P, Mode::CHEBLAST, ADJ>(a, st);
    }
    set_error("mode not available for the element-parallel kernels");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
jfnk_status launch_ep3d(Prob prob, Mode mode, bool adj, const StencilArgs<T>& a, cudaStream_t st) {
    if (prob == Prob::ND3)
        return adj ? launch_ep3d_p<T, Prob::ND3, true>(mode, a, st) : launch_ep3d_p<T, Prob::ND3, false>(mode, a, st);
    if (prob == Prob::NDK3)
        return adj ? launch_ep3d_p<T, Prob::NDK3, true>(mode, a, st)
                   : launch_ep3d_p<T, Prob::NDK3, false>(mode, a, st);
    set_error("the element-parallel kernels are 3D only");
    return JFNK_ERR_INVALID_ARG;
}

template jfnk_status launch_ep3d<double>(Prob, Mode, bool, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_ep3d<float>(Prob, Mode, bool, const StencilArgs<float>&, cudaStream_t);

}  // namespace jfnk
