// Kernels of the hyperelastic beam (Sec. 3, "Hyperelasticity"): 10n x n x n
// cube elements, three displacement components per node (component fastest),
// Dirichlet data on the faces x = 0 and x = 10, free lateral faces.
//
// Element residual: the same element-parallel design as the 3D scalar
// problems -- one thread per element forms w = x + eps v at its 8 corners
// (direction entries on the Dirichlet faces ignored), evaluates the
// Neo-Hookean element and stores its 24 contributions in scratch; one thread
// per node sums the contributions of the (up to 8) elements around it in a
// fixed order and applies the fused epilogue of the mode to each component;
// the last block completes the norm reduction.
//
// Transfers (Sec. 2): R = I^T, I the trilinear interpolation of corrections
// (zero on the Dirichlet faces), and the projection of the iterate
// I^T x / (I^T 1) -- each row divided by its weight sum, which is 2^3 away from
// the free faces (the paper's 2^-d I^T) and keeps constants on them -- with the
// Dirichlet data injected.
#include <algorithm>

#include "beam.cuh"
#include "element.cuh"
#include "reduce.cuh"
#include "stencil_body.cuh"

namespace jfnk {

constexpr int kBeamElemThreads = 128;
constexpr int kBeamNodeThreads = 128;

template <typename T, Mode M>
__global__ void __launch_bounds__(kBeamElemThreads) beam_elem_kernel(const StencilArgs<T> a) {
    const Grid g = a.g;
    const int ex = 10 * g.n, ey = g.n, ez = g.n;
    const long long ne = (long long)ex * ey * ez;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= ex) return;
    T eps = T(0);
    if (M != Mode::F) eps = eps_of<T>(a.eps);
    T ue[24];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int X = x + (c & 1), Y = y + ((c >> 1) & 1), Z = z + (c >> 2);
        const long long node = ((long long)Z * g.ny + Y) * g.nx + X;
        const bool dir = X == 0 || X == g.nx - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T val = a.u[node * 3 + i];
            if (M != Mode::F && !dir) val += eps * a.v[node * 3 + i];
            ue[3 * c + i] = val;
        }
    }
    T r[24];
    elem_neohooke<T>(ue, a.lh, r);
    const long long e = ((long long)z * ey + y) * ex + x;
    T* C = a.face + e;
#pragma unroll
    for (int k = 0; k < 24; ++k) C[k * ne] = r[k];
}

template <typename T, Mode M>
__global__ void __launch_bounds__(kBeamNodeThreads) beam_node_kernel(const StencilArgs<T> a) {
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int ex = 10 * g.n, ey = g.n, ez = g.n;
    const long long ne = (long long)ex * ey * ez;
    const T* C = a.face;
    T inv_eps = T(0);
    if (M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    for (int row = blockIdx.x; row < g.ny * g.nz; row += gridDim.x) {
        const int Y = row % g.ny, Z = row / g.ny;
        for (int X = threadIdx.x; X < g.nx; X += blockDim.x) {
            const long long node = ((long long)Z * g.ny + Y) * g.nx + X;
            const bool inner = X > 0 && X < g.nx - 1;
            T val[3] = {T(0), T(0), T(0)};
            if (inner) {
                // element with corner c at this node: (X - dx, Y - dy, Z - dz), fixed order c = 0..7
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int xe = X - (c & 1), ye = Y - ((c >> 1) & 1), ze = Z - (c >> 2);
                    if (xe < 0 || xe >= ex || ye < 0 || ye >= ey || ze < 0 || ze >= ez) continue;
                    const long long e = ((long long)ze * ey + ye) * ex + xe;
#pragma unroll
                    for (int i = 0; i < 3; ++i) val[i] += C[(3 * c + i) * ne + e];
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) epilogue<T, M>(a, node * 3 + i, inner, val[i], inv_eps, ck, red);
        }
    }
    stencil_reduce(a, red, red_sm);
}

template <typename T, Mode M>
static jfnk_status launch_beam_m(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    if (!g.beam || g.n < 1 || g.n > 256) {
        set_error("beam kernels: not a beam grid, or n = %d outside [1, 256]", g.n);
        return JFNK_ERR_INVALID_ARG;
    }
    if (beam_scratch_count(g) > a.face_cap || !a.face) {
        set_error("beam element scratch too small (%lld < %lld)", a.face_cap, beam_scratch_count(g));
        return JFNK_ERR_WORKSPACE;
    }
    const int ex = 10 * g.n;
    const int bx = std::min(kBeamElemThreads, ((ex + 31) / 32) * 32);
    beam_elem_kernel<T, M><<<dim3((ex + bx - 1) / bx, g.n, g.n), bx, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    const int nb = std::min(g.ny * g.nz, 2 * kMaxRedBlocks);
    beam_node_kernel<T, M><<<nb, kBeamNodeThreads, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T>
jfnk_status launch_beam(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::F: return launch_beam_m<T, Mode::F>(a, st);
        case Mode::JV: return launch_beam_m<T, Mode::JV>(a, st);
        case Mode::BMJ: return launch_beam_m<T, Mode::BMJ>(a, st);
        case Mode::CHEB0: return launch_beam_m<T, Mode::CHEB0>(a, st);
        case Mode::CHEB: return launch_beam_m<T, Mode::CHEB>(a, st);
        case Mode::CHEBLAST: return launch_beam_m<T, Mode::CHEBLAST>(a, st);
    }
    set_error("unknown stencil mode");
    return JFNK_ERR_INVALID_ARG;
}
template jfnk_status launch_beam<double>(Mode, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_beam<float>(Mode, const StencilArgs<float>&, cudaStream_t);

// ---------------------------------------------------------------------------
// Transfers
// ---------------------------------------------------------------------------
// Coarse entry (X, Y, Z, i) gathers the fine nodes (2X+a, 2Y+b, 2Z+c), a, b, c in
// {-1, 0, 1}, with weights 1 (0) and 1/2 (+-1) per axis.
template <typename T>
__global__ void beam_restrict_kernel(Grid gc, Grid gf, const T* __restrict__ f, T* __restrict__ c, int projection) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < gc.size;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % 3);
        const long long node = k / 3;
        const int X = (int)(node % gc.nx);
        const long long yz = node / gc.nx;
        const int Y = (int)(yz % gc.ny), Z = (int)(yz / gc.ny);
        const bool cdir = X == 0 || X == gc.nx - 1;
        if (cdir) {
            c[k] = projection ? f[((((long long)2 * Z) * gf.ny + 2 * Y) * gf.nx + 2 * X) * 3 + i] : T(0);
            continue;
        }
        double acc = 0.0, wsum = 0.0;
        for (int dz = -1; dz <= 1; ++dz) {
            const int zf = 2 * Z + dz;
            if (zf < 0 || zf >= gf.nz) continue;
            const double wz = dz == 0 ? 1.0 : 0.5;
            for (int dy = -1; dy <= 1; ++dy) {
                const int yf = 2 * Y + dy;
                if (yf < 0 || yf >= gf.ny) continue;
                const double wy = dy == 0 ? 1.0 : 0.5;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xf = 2 * X + dx;  // 1 <= xf <= gf.nx - 2 for an interior coarse node
                    const double w = wz * wy * (dx == 0 ? 1.0 : 0.5);
                    const bool fdir = xf == 0 || xf == gf.nx - 1;
                    const double fv = (!projection && fdir) ? 0.0 : (double)f[(((long long)zf * gf.ny + yf) * gf.nx + xf) * 3 + i];
                    acc += w * fv;
                    wsum += w;
                }
            }
        }
        c[k] = (T)(projection ? acc / wsum : acc);
    }
}

// Fine entry += trilinear interpolation of the coarse correction (coarse
// Dirichlet entries taken as 0); fine Dirichlet entries untouched.
template <typename T>
__global__ void beam_prolong_add_kernel(Grid gf, Grid gc, const T* __restrict__ c, T* __restrict__ s) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < gf.size;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % 3);
        const long long node = k / 3;
        const int x = (int)(node % gf.nx);
        const long long yz = node / gf.nx;
        const int y = (int)(yz % gf.ny), z = (int)(yz / gf.ny);
        if (x == 0 || x == gf.nx - 1) continue;
        const int x0 = x >> 1, x1 = (x + 1) >> 1, y0 = y >> 1, y1 = (y + 1) >> 1, z0 = z >> 1, z1 = (z + 1) >> 1;
        const double wx = (x & 1) ? 0.5 : 1.0, wy = (y & 1) ? 0.5 : 1.0, wz = (z & 1) ? 0.5 : 1.0;
        double acc = 0.0;
        for (int cz = 0; cz < ((z & 1) ? 2 : 1); ++cz)
            for (int cy = 0; cy < ((y & 1) ? 2 : 1); ++cy)
                for (int cx = 0; cx < ((x & 1) ? 2 : 1); ++cx) {
                    const int X = cx ? x1 : x0, Y = cy ? y1 : y0, Z = cz ? z1 : z0;
                    if (X == 0 || X == gc.nx - 1) continue;
                    acc += wx * wy * wz * (double)c[(((long long)Z * gc.ny + Y) * gc.nx + X) * 3 + i];
                }
        s[k] += (T)acc;
    }
}

template <typename T>
jfnk_status beam_restrict(const Grid& gf, const Grid& gc, const T* f, T* c, bool projection, cudaStream_t st) {
    const long long b = std::min<long long>((gc.size + 255) / 256, 4096);
    beam_restrict_kernel<T><<<(int)std::max<long long>(b, 1), 256, 0, st>>>(gc, gf, f, c, projection ? 1 : 0);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template <typename T>
jfnk_status beam_prolong_add(const Grid& gc, const Grid& gf, const T* c, T* s, cudaStream_t st) {
    const long long b = std::min<long long>((gf.size + 255) / 256, 4096);
    beam_prolong_add_kernel<T><<<(int)std::max<long long>(b, 1), 256, 0, st>>>(gf, gc, c, s);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status beam_restrict<double>(const Grid&, const Grid&, const double*, double*, bool, cudaStream_t);
template jfnk_status beam_restrict<float>(const Grid&, const Grid&, const float*, float*, bool, cudaStream_t);
template jfnk_status beam_prolong_add<double>(const Grid&, const Grid&, const double*, double*, cudaStream_t);
template jfnk_status beam_prolong_add<float>(const Grid&, const Grid&, const float*, float*, cudaStream_t);

}  // namespace jfnk
