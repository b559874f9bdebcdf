// Adjoint operator: hand-written vector-Jacobian product of the element
// residual of the nonlinear-diffusion problems,
//   (J^T v)_b = sum_e kappa_e int_e (1+u^2) grad v . grad phi_b + 2 u (grad u . grad v) phi_b
//   (dF/dkappa_e)^T v = int_e (1+u^2) grad u . grad v,
// with the same tiling as the forward tiled kernel (32 x 8 threads, 31 x 7 node
// columns per CTA, z march, both fields staged in shared memory) and the same
// fused epilogues (b - J^T v, Chebyshev start/step) so that the multigrid
// cycle of Algorithm 1 can be run on J^T for the adjoint solve.  J^T v is
// exact here (no FD step): the adjoint of a Jacobian-free forward solve is
// defined by the true Jacobian.
#include <algorithm>

#include "element.cuh"
#include "reduce.cuh"
#include "stencil.cuh"
#include "stencil_body.cuh"
#include "stencil_ep.cuh"

namespace jfnk {

constexpr int KA_BX = 32, KA_BY = 8, KA_TX = KA_BX - 1, KA_TY = KA_BY - 1;
constexpr int KA_WX = KA_BX + 1, KA_WY = KA_BY + 1;

template <typename T, bool KAPPA, Mode M>
__global__ void __launch_bounds__(KA_BX* KA_BY) vjp3d_kernel(const StencilArgs<T> a, int zchunk) {
    __shared__ T U[2][KA_WY][KA_WX];
    __shared__ T V[2][KA_WY][KA_WX];
    __shared__ T C[8][KA_BY][KA_BX];
    __shared__ double red_sm[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * KA_BX + tx;
    const Grid g = a.g;
    const int n = g.n;
    const int x0 = blockIdx.x * KA_TX, y0 = blockIdx.y * KA_TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
    const bool elem_xy = ex >= 0 && ex < n && ey >= 0 && ey < n;
    const int nx_o = x0 + tx, ny_o = y0 + ty;
    const bool node_thr = tx < KA_TX && ty < KA_TY && nx_o < g.nx && ny_o < g.ny;
    const bool inner_xy = nx_o > 0 && nx_o < g.nx - 1 && ny_o > 0 && ny_o < g.ny - 1;
    // the element is written by the CTA that owns its lower corner node
    const bool own_elem = elem_xy && tx >= 1 && ty >= 1;

    auto load_plane = [&](int z, int buf) {
        for (int i = tid; i < KA_WX * KA_WY; i += KA_BX * KA_BY) {
            const int lx = i % KA_WX, ly = i / KA_WX;
            const int x = x0 - 1 + lx, y = y0 - 1 + ly;
            T uv = T(0), vv = T(0);
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
                const long long idx = (long long)z * g.sz + (long long)y * g.sy + x;
                uv = a.u[idx];
                const bool bnd = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1;
                if (!bnd) vv = a.v[idx];
            }
            U[buf][ly][lx] = uv;
            V[buf][ly][lx] = vv;
        }
    };

    T carry = T(0);
    float red = 0.f;
    const T scale = a.node_scale;
    load_plane(z0 - 1, (z0 - 1) & 1);
    for (int k = z0 - 1; k < z1; ++k) {
        load_plane(k + 1, (k + 1) & 1);
        __syncthreads();
        T r[8];
        if (elem_xy && k >= 0 && k < n) {
            const int b0 = k & 1, b1 = (k + 1) & 1;
            T ue[8] = {U[b0][ty][tx], U[b0][ty][tx + 1], U[b0][ty + 1][tx], U[b0][ty + 1][tx + 1],
                       U[b1][ty][tx], U[b1][ty][tx + 1], U[b1][ty + 1][tx], U[b1][ty + 1][tx + 1]};
            T ve[8] = {V[b0][ty][tx], V[b0][ty][tx + 1], V[b0][ty + 1][tx], V[b0][ty + 1][tx + 1],
                       V[b1][ty][tx], V[b1][ty][tx + 1], V[b1][ty + 1][tx], V[b1][ty + 1][tx + 1]};
            const long long e = ((long long)k * n + ey) * n + ex;
            const T kap = KAPPA ? a.kappa[e] : T(1);
            T dk;
            elem_vjp3<T>(ue, ve, kap, r, dk);
            if (a.dkout && own_elem && k >= z0) a.dkout[e] = dk * a.dk_scale;
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
                epilogue_adj<T, M>(a, idx, inner, (carry + lower) * scale, ck, red);
            }
            carry = upper;
        }
    }
    if (a.red == RedOut::NONE) return;
    double bs = block_sum(red, red_sm);
    double tot = 0.0;
    if (grid_sum_last(bs, a.partials, a.counter, &tot, red_sm)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double nrm = sqrt(tot);
            if (a.red_norm) *a.red_norm = nrm;
            if (a.red == RedOut::EPS) {  // keeps the FD-step slot meaningful for mixed use
                double e = eps_formula(a.epsp.mode, a.epsp.n_unknowns, *a.epsp.xstat, nrm);
                double inv = e > 0.0 ? 1.0 / e : 0.0;
                a.red_eps->e = e;
                a.red_eps->inv = inv;
                a.red_eps->ef = (float)e;
                a.red_eps->invf = (float)inv;
            }
        }
    }
}

template <typename T, bool KAPPA, Mode M>
static jfnk_status launch_vjp_km(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    const int gx = (g.nx + KA_TX - 1) / KA_TX, gy = (g.ny + KA_TY - 1) / KA_TY;
    const long long tiles = (long long)gx * gy;
    long long chunks = std::max<long long>(1, (152LL * 6) / std::max<long long>(1, tiles));
    int zc = (int)((g.nz + chunks - 1) / chunks);
    zc = std::min(std::max(zc, 8), g.nz);
    const int gz = (g.nz + zc - 1) / zc;
    if (tiles * gz > kMaxRedBlocks * 2) {
        set_error("adjoint grid too large for the reduction scratch");
        return JFNK_ERR_INVALID_ARG;
    }
    vjp3d_kernel<T, KAPPA, M><<<dim3(gx, gy, gz), dim3(KA_BX, KA_BY), 0, st>>>(a, zc);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, bool KAPPA>
static jfnk_status launch_vjp_k(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::JV: return launch_vjp_km<T, KAPPA, Mode::JV>(a, st);
        case Mode::BMJ: return launch_vjp_km<T, KAPPA, Mode::BMJ>(a, st);
        case Mode::CHEB0: return launch_vjp_km<T, KAPPA, Mode::CHEB0>(a, st);
        case Mode::CHEB: return launch_vjp_km<T, KAPPA, Mode::CHEB>(a, st);
        case Mode::CHEBLAST: return launch_vjp_km<T, KAPPA, Mode::CHEBLAST>(a, st);
        default: break;
    }
    set_error("mode not available for the adjoint operator");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
jfnk_status launch_vjp(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    if ((prob == Prob::NDK3 || prob == Prob::ND3) && ep3d_use(a, true)) return launch_ep3d<T>(prob, mode, true, a, st);
    if (prob == Prob::NDK3) return launch_vjp_k<T, true>(mode, a, st);
    if (prob == Prob::ND3) return launch_vjp_k<T, false>(mode, a, st);
    set_error("the adjoint operator is implemented for the 3D diffusion problems");
    return JFNK_ERR_NOT_IMPLEMENTED;
}

template jfnk_status launch_vjp<double>(Prob, Mode, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_vjp<float>(Prob, Mode, const StencilArgs<float>&, cudaStream_t);

}  // namespace jfnk
