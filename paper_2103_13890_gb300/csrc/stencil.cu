// Tiled Q1 residual kernels F(w), w = x + eps v, with fused epilogues.
//
// 3D: a CTA of 32 x 8 threads owns an output tile of 31 x 7 node columns and
// marches along z.  Thread (tx, ty) evaluates the element whose lower corner
// is node (x0-1+tx, y0-1+ty) on every layer; node planes are staged in shared
// memory (one halo node on the low side and one on the high side in x and y)
// and element contributions are exchanged through shared memory, so each node
// sums its 2^d element contributions in a fixed order (deterministic).  The
// contribution of a layer to the plane above is carried in a register.
// 2D: a CTA of BX threads owns a row segment of BX-1 nodes and marches along y.
//
// Every element integral is the one of the problem definition (element.cuh);
// F is assembled node by node, so the kernels are exact restatements of
// F_i = sum_e int_e ..., with Dirichlet rows set to zero.
#include <algorithm>
#include <cstdio>

#include "element.cuh"
#include "profile.cuh"
#include "stencil_body.cuh"
#include "stencil_ep.cuh"
#include "beam.cuh"
#include "stencil_v2.cuh"
#include "reduce.cuh"
#include "stencil.cuh"

namespace jfnk {

// ---------------------------------------------------------------------------
// 3D kernel
// ---------------------------------------------------------------------------
constexpr int K3_BX = 32, K3_BY = 8, K3_TX = K3_BX - 1, K3_TY = K3_BY - 1;
constexpr int K3_WX = K3_BX + 1, K3_WY = K3_BY + 1;

template <typename T, Prob P, Mode M>
__global__ void __launch_bounds__(K3_BX* K3_BY) stencil3d_kernel(const StencilArgs<T> a, int zchunk) {
    __shared__ T W[2][K3_WY][K3_WX];
    __shared__ T C[8][K3_BY][K3_BX];
    __shared__ double red_sm[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * K3_BX + tx;
    const Grid g = a.g;
    const int n = g.n;
    const int x0 = blockIdx.x * K3_TX, y0 = blockIdx.y * K3_TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    T eps = T(0), inv_eps = T(0);
    if (M != Mode::F) {
        eps = eps_of<T>(a.eps);
        inv_eps = inv_eps_of<T>(a.eps);
    }
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);

    const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
    const bool elem_xy = ex >= 0 && ex < n && ey >= 0 && ey < n;
    const int nx_o = x0 + tx, ny_o = y0 + ty;
    const bool node_thr = tx < K3_TX && ty < K3_TY && nx_o < g.nx && ny_o < g.ny;
    const bool inner_xy = nx_o > 0 && nx_o < g.nx - 1 && ny_o > 0 && ny_o < g.ny - 1;

    auto load_plane = [&](int z, int buf) {
        for (int i = tid; i < K3_WX * K3_WY; i += K3_BX * K3_BY) {
            const int lx = i % K3_WX, ly = i / K3_WX;
            const int x = x0 - 1 + lx, y = y0 - 1 + ly;
            T val = T(0);
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
                const long long idx = JFNK_IDX((long long)z * g.sz + (long long)y * g.sy + x, g.size);
                val = a.u[idx];
                if (M != Mode::F) {
                    const bool bnd = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1;
                    if (!bnd) val += eps * a.v[idx];
                }
            }
            W[buf][ly][lx] = val;
        }
    };

    T carry = T(0);
    float red = 0.f;
    load_plane(z0 - 1, (z0 - 1) & 1);
    for (int k = z0 - 1; k < z1; ++k) {
        load_plane(k + 1, (k + 1) & 1);
        __syncthreads();
        T r[8];
        if (elem_xy && k >= 0 && k < n) {
            const int b0 = k & 1, b1 = (k + 1) & 1;
            T ue[8] = {W[b0][ty][tx],     W[b0][ty][tx + 1],     W[b0][ty + 1][tx],     W[b0][ty + 1][tx + 1],
                       W[b1][ty][tx],     W[b1][ty][tx + 1],     W[b1][ty + 1][tx],     W[b1][ty + 1][tx + 1]};
            if (P == Prob::NDK3)
                elem_nd3<T, true>(ue, a.kappa[JFNK_IDX(((long long)k * n + ey) * n + ex, (long long)n * n * n)], r);
            else
                elem_nd3<T, false>(ue, T(1), r);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) r[c] = T(0);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) C[c][ty][tx] = r[c];
        __syncthreads();
        if (node_thr) {
            const T lower = C[3][ty][tx] + C[2][ty][tx + 1] + C[1][ty + 1][tx] + C[0][ty + 1][tx + 1];
            const T upper = C[7][ty][tx] + C[6][ty][tx + 1] + C[5][ty + 1][tx] + C[4][ty + 1][tx + 1];
            if (k >= z0) {
                const long long idx = (long long)k * g.sz + (long long)ny_o * g.sy + nx_o;
                const bool inner = inner_xy && k > 0 && k < g.nz - 1;
                epilogue<T, M>(a, idx, inner, (carry + lower) * a.node_scale, inv_eps, ck, red);
            }
            carry = upper;
        }
    }
    stencil_reduce(a, red, red_sm);
}

// ---------------------------------------------------------------------------
// 2D kernel (Bratu), blockDim.x = BX threads, BX-1 output nodes per row segment
// ---------------------------------------------------------------------------
template <typename T, Prob P, Mode M>
__global__ void __launch_bounds__(512) stencil2d_kernel(const StencilArgs<T> a, int ychunk, int txo) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ double red_sm[32];
    const int y0 = blockIdx.y * ychunk;
    stencil2d_body<T, M, P>(a, blockIdx.x * txo, y0, min(y0 + ychunk, a.g.ny), txo, blockIdx.x + gridDim.x * blockIdx.y,
                         gridDim.x * gridDim.y, smem_raw, red_sm);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int chunk_for(long long tiles, int extent, int min_chunk) {
    // aim for a few waves of CTAs over the 152 SMs
    const long long target = 152LL * 6;
    long long chunks = std::max<long long>(1, target / std::max<long long>(1, tiles));
    int chunk = (int)((extent + chunks - 1) / chunks);
    chunk = std::max(chunk, min_chunk);
    return std::min(chunk, extent);
}

template <typename T, Prob P, Mode M>
static jfnk_status launch3(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    const int gx = (g.nx + K3_TX - 1) / K3_TX, gy = (g.ny + K3_TY - 1) / K3_TY;
    const int zc = chunk_for((long long)gx * gy, g.nz, 8);
    const int gz = (g.nz + zc - 1) / zc;
    if ((long long)gx * gy * gz > kMaxRedBlocks * 2) {
        set_error("3D grid too large for the reduction scratch (%d x %d x %d)", gx, gy, gz);
        return JFNK_ERR_INVALID_ARG;
    }
    stencil3d_kernel<T, P, M><<<dim3(gx, gy, gz), dim3(K3_BX, K3_BY), 0, st>>>(a, zc);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, Prob P, Mode M>
static jfnk_status launch2(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    // row segments of txo nodes: fewest segments with <= 511 nodes each
    int segs = (g.nx + 510) / 511;
    int txo = (g.nx + segs - 1) / segs;
    int bx = ((txo + 1 + 31) / 32) * 32;
    const int yc = chunk_for(segs, g.ny, 4);
    const int gy = (g.ny + yc - 1) / yc;
    if ((long long)segs * gy > kMaxRedBlocks * 2) {
        set_error("2D grid too large for the reduction scratch");
        return JFNK_ERR_INVALID_ARG;
    }
    size_t smem = sizeof(T) * (2 * (bx + 1) + 4 * bx);
    stencil2d_kernel<T, P, M><<<dim3(segs, gy), dim3(bx), smem, st>>>(a, yc, txo);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, Prob P>
static jfnk_status dispatch_mode(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    if constexpr (is_2d(P)) {
        switch (mode) {
            case Mode::F: return launch2<T, P, Mode::F>(a, st);
            case Mode::JV: return launch2<T, P, Mode::JV>(a, st);
            case Mode::BMJ: return launch2<T, P, Mode::BMJ>(a, st);
            case Mode::CHEB0: return launch2<T, P, Mode::CHEB0>(a, st);
            case Mode::CHEB: return launch2<T, P, Mode::CHEB>(a, st);
            case Mode::CHEBLAST: return launch2<T, P, Mode::CHEBLAST>(a, st);
        }
    } else {
        switch (mode) {
            case Mode::F: return launch3<T, P, Mode::F>(a, st);
            case Mode::JV: return launch3<T, P, Mode::JV>(a, st);
            case Mode::BMJ: return launch3<T, P, Mode::BMJ>(a, st);
            case Mode::CHEB0: return launch3<T, P, Mode::CHEB0>(a, st);
            case Mode::CHEB: return launch3<T, P, Mode::CHEB>(a, st);
            case Mode::CHEBLAST: return launch3<T, P, Mode::CHEBLAST>(a, st);
        }
    }
    set_error("unknown stencil mode");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
static jfnk_status launch_stencil_impl(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    if (prob == Prob::BEAM3) return launch_beam<T>(mode, a, st);
    if (!is_2d(prob) && ep3d_use(a)) return launch_ep3d<T>(prob, mode, false, a, st);
    if (!is_2d(prob) && a.face != nullptr && a.v2_threads >= 0 && v2_applicable(a.g)) {
        if constexpr (sizeof(T) == 4) {
            if (a.v3) return launch_stencil_v3(prob, mode, a, st);
        }
        return launch_stencil_v2<T>(prob, mode, a, st);
    }
    switch (prob) {
        case Prob::BRATU2: return dispatch_mode<T, Prob::BRATU2>(mode, a, st);
        case Prob::MINSURF2: return dispatch_mode<T, Prob::MINSURF2>(mode, a, st);
        case Prob::BEAM3: break;
        case Prob::ND3: return dispatch_mode<T, Prob::ND3>(mode, a, st);
        case Prob::NDK3: return dispatch_mode<T, Prob::NDK3>(mode, a, st);
    }
    set_error("unknown problem kind");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
jfnk_status launch_stencil(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    if (!prof_on()) return launch_stencil_impl<T>(prob, mode, a, st);
    static const char* pn[] = {"bratu2d", "nd3d", "ndk3d", "minsurf2d", "beam3d"};
    static const char* mn[] = {"F", "JV", "BMJ", "CHEB0", "CHEB", "CHEBLAST"};
    char name[96];
    snprintf(name, sizeof(name), "stencil_%s_%s_%s_n%d", pn[(int)prob], sizeof(T) == 8 ? "f64" : "f32",
             mn[(int)mode], a.g.n);
    const double elems = (double)a.g.elements();
    prof_begin(name, elems, st);
    jfnk_status s = launch_stencil_impl<T>(prob, mode, a, st);
    prof_end(st);
    return s;
}

// Launch without the optional event profiler (which creates CUDA events).
template <typename T>
jfnk_status launch_stencil_direct(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    return launch_stencil_impl<T>(prob, mode, a, st);
}
template jfnk_status launch_stencil_direct<double>(Prob, Mode, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_stencil_direct<float>(Prob, Mode, const StencilArgs<float>&, cudaStream_t);

template jfnk_status launch_stencil<double>(Prob, Mode, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_stencil<float>(Prob, Mode, const StencilArgs<float>&, cudaStream_t);

}  // namespace jfnk
