// Transfer operators between nested structured Q1 grids (Sec. 2, "Transfer
// Operators"): interpolation I (coarse -> fine), restriction R = I^T and the
// projection of the Newton iterate P = 2^-d I^T.  Coarse node i coincides with
// fine node 2i; in 1D, I puts c_i on fine node 2i and (c_i + c_(i+1))/2 on fine
// node 2i+1, and the d-dimensional I is the tensor product.
//
// The fine neighbours 2i-1, 2i, 2i+1 of an interior coarse node are interior
// fine nodes, so R and P read interior values only; coarse boundary entries
// are 0 for R and the injected Dirichlet value for P.
#include "transfer.cuh"
#include "beam.cuh"

namespace jfnk {

constexpr int kTThreads = 256;

static int t_blocks(long long n) {
    long long b = (n + kTThreads - 1) / kTThreads;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

// c[I] = scale * sum_{o in {-1,0,1}^d} w(o) f[2I + o],  w(o) = prod (o == 0 ? 1 : 1/2)
template <typename T>
__global__ void restrict_kernel(Grid gc, Grid gf, const T* __restrict__ f, T* __restrict__ c, T scale,
                                int inject_boundary) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < gc.size;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        grid_coords(gc, i, x, y, z);
        const bool bnd = x == 0 || x == gc.nx - 1 || y == 0 || y == gc.ny - 1 ||
                         (gc.d == 3 && (z == 0 || z == gc.nz - 1));
        const long long fc = JFNK_IDX((gc.d == 3 ? (long long)(2 * z) * gf.sz : 0) + (long long)(2 * y) * gf.sy + 2 * x,
                                      gf.size);
        if (bnd) {
            c[i] = inject_boundary ? f[fc] : T(0);
            continue;
        }
        // the 3^d fine neighbours of an interior coarse node
        (void)JFNK_IDX(fc - (gc.d == 3 ? gf.sz : 0) - gf.sy - 1, gf.size);
        (void)JFNK_IDX(fc + (gc.d == 3 ? gf.sz : 0) + gf.sy + 1, gf.size);
        T acc = T(0);
        if (gc.d == 2) {
#pragma unroll
            for (int oy = -1; oy <= 1; ++oy) {
                T row = T(0.5) * (f[fc + oy * gf.sy - 1] + f[fc + oy * gf.sy + 1]) + f[fc + oy * gf.sy];
                acc += (oy == 0 ? T(1) : T(0.5)) * row;
            }
        } else {
#pragma unroll
            for (int oz = -1; oz <= 1; ++oz) {
                T pl = T(0);
#pragma unroll
                for (int oy = -1; oy <= 1; ++oy) {
                    const long long b = fc + oz * gf.sz + oy * gf.sy;
                    T row = T(0.5) * (f[b - 1] + f[b + 1]) + f[b];
                    pl += (oy == 0 ? T(1) : T(0.5)) * row;
                }
                acc += (oz == 0 ? T(1) : T(0.5)) * pl;
            }
        }
        c[i] = scale * acc;
    }
}

template <typename T>
jfnk_status restrict_to(const Grid& gf, const Grid& gc, const T* f, T* c, bool projection, cudaStream_t st) {
    if (gf.beam) return beam_restrict<T>(gf, gc, f, c, projection, st);
    const T scale = projection ? (gc.d == 3 ? T(0.125) : T(0.25)) : T(1);
    restrict_kernel<T><<<t_blocks(gc.size), kTThreads, 0, st>>>(gc, gf, f, c, scale, projection ? 1 : 0);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

// s_f += I c on interior fine nodes (coarse boundary entries taken as 0)
template <typename T>
__global__ void prolong_add_kernel(Grid gf, Grid gc, const T* __restrict__ c, T* __restrict__ s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < gf.size;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        grid_coords(gf, i, x, y, z);
        const bool bnd = x == 0 || x == gf.nx - 1 || y == 0 || y == gf.ny - 1 ||
                         (gf.d == 3 && (z == 0 || z == gf.nz - 1));
        if (bnd) continue;
        // per direction: coarse indices and weights
        int ix[2], iy[2], iz[2];
        T wx[2], wy[2], wz[2];
        int nxs = 1, nys = 1, nzs = 1;
        if (x & 1) { ix[0] = x >> 1; ix[1] = (x >> 1) + 1; wx[0] = wx[1] = T(0.5); nxs = 2; }
        else { ix[0] = x >> 1; wx[0] = T(1); }
        if (y & 1) { iy[0] = y >> 1; iy[1] = (y >> 1) + 1; wy[0] = wy[1] = T(0.5); nys = 2; }
        else { iy[0] = y >> 1; wy[0] = T(1); }
        if (gf.d == 3 && (z & 1)) { iz[0] = z >> 1; iz[1] = (z >> 1) + 1; wz[0] = wz[1] = T(0.5); nzs = 2; }
        else { iz[0] = (gf.d == 3) ? (z >> 1) : 0; wz[0] = T(1); }
        T acc = T(0);
        for (int a = 0; a < nzs; ++a) {
            const bool zb = gf.d == 3 && (iz[a] == 0 || iz[a] == gc.nz - 1);
            for (int b = 0; b < nys; ++b) {
                const bool yb = iy[b] == 0 || iy[b] == gc.ny - 1;
                for (int q = 0; q < nxs; ++q) {
                    const bool xb = ix[q] == 0 || ix[q] == gc.nx - 1;
                    if (zb || yb || xb) continue;
                    acc += wz[a] * wy[b] * wx[q] *
                           c[JFNK_IDX((long long)iz[a] * gc.sz + (long long)iy[b] * gc.sy + ix[q], gc.size)];
                }
            }
        }
        s[i] += acc;
    }
}

template <typename T>
jfnk_status prolong_add(const Grid& gc, const Grid& gf, const T* c, T* s, cudaStream_t st) {
    if (gf.beam) return beam_prolong_add<T>(gc, gf, c, s, st);
    prolong_add_kernel<T><<<t_blocks(gf.size), kTThreads, 0, st>>>(gf, gc, c, s);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template jfnk_status restrict_to<float>(const Grid&, const Grid&, const float*, float*, bool, cudaStream_t);
template jfnk_status restrict_to<double>(const Grid&, const Grid&, const double*, double*, bool, cudaStream_t);
template jfnk_status prolong_add<float>(const Grid&, const Grid&, const float*, float*, cudaStream_t);
template jfnk_status prolong_add<double>(const Grid&, const Grid&, const double*, double*, cudaStream_t);

// per-element coefficient of the coarse grid: mean of the 2^d children
__global__ void coarsen_kappa_kernel(int nc, const double* __restrict__ kf, double* __restrict__ kc) {
    const long long tot = (long long)nc * nc * nc;
    const int nf = 2 * nc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nc), y = (int)((i / nc) % nc), z = (int)(i / ((long long)nc * nc));
        double acc = 0.0;
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a)
                    acc += kf[((long long)(2 * z + c) * nf + (2 * y + b)) * nf + (2 * x + a)];
        kc[i] = acc * 0.125;
    }
}

jfnk_status coarsen_kappa(int nc, const double* kf, double* kc, cudaStream_t st) {
    coarsen_kappa_kernel<<<t_blocks((long long)nc * nc * nc), kTThreads, 0, st>>>(nc, kf, kc);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

// Manufactured load b_i = int f phi_i for f = -div((1+u*^2) grad u*),
// u* = sin(pi x) sin(pi y) sin(pi z).  f is a sum of five separable products
//   f = 3pi^2 s s s + 3pi^2 s^3 s^3 s^3 - 2pi^2 (s c^2 s^3 s^3 + s^3 s c^2 s^3 + s^3 s^3 s c^2)
// (s = sin(pi .), c = cos(pi .)), and the 3-point tensor Gauss rule of a
// separable integrand against a tensor-product hat function factorises, so
// b_ijk = 3pi^2 I1_i I1_j I1_k + 3pi^2 I3_i I3_j I3_k
//         - 2pi^2 (Ic_i I3_j I3_k + I3_i Ic_j I3_k + I3_i I3_j Ic_k)
// with 1D tables I1 = int s hat_i, I3 = int s^3 hat_i, Ic = int s c^2 hat_i.
__global__ void mms_load_kernel(Grid g, const double* __restrict__ tab, double* __restrict__ b) {
    const int np = g.nx;
    const double* I1 = tab;
    const double* I3 = tab + np;
    const double* Ic = tab + 2 * np;
    const double pi2 = 9.869604401089358;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.size;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        grid_coords(g, i, x, y, z);
        const bool bnd = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1;
        double v = 0.0;
        if (!bnd) {
            v = 3.0 * pi2 * (I1[x] * I1[y] * I1[z] + I3[x] * I3[y] * I3[z]) -
                2.0 * pi2 * (Ic[x] * I3[y] * I3[z] + I3[x] * Ic[y] * I3[z] + I3[x] * I3[y] * Ic[z]);
        }
        b[i] = v;
    }
}

jfnk_status mms_load(const Grid& g, const double* tab_dev, double* b, cudaStream_t st) {
    mms_load_kernel<<<t_blocks(g.size), kTThreads, 0, st>>>(g, tab_dev, b);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

}  // namespace jfnk
