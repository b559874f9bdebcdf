// Vector kernels: deterministic reductions (fixed grids, last-block
// completion), BLAS-1 updates, casts and the power-method start vector.
#include "reduce.cuh"
#include "vector.cuh"

namespace jfnk {

constexpr int kVecThreads = 256;
// 8 x 152 SMs: every SM holds 2048 threads, so the streaming kernels keep
// enough loads in flight to reach HBM speed (at 2 x 152 blocks a one-load-per-
// iteration loop ran at ~0.6 TB/s); fixed, so sums are reproducible, and
// within the 2 kMaxRedBlocks reduction partials
constexpr int kVecBlocks = 1216;
static_assert(kVecBlocks <= 2 * kMaxRedBlocks, "reduction partials");

// about 8 entries a thread (loads in flight without a long tail of per-block
// completions on short vectors), at most kVecBlocks blocks
static int vec_blocks(long long len) {
    long long b = (len + 8 * kVecThreads - 1) / (8 * kVecThreads);
    return (int)(b < kVecBlocks ? (b < 1 ? 1 : b) : kVecBlocks);
}

__device__ __forceinline__ bool grid_inner(const Grid& g, long long i) { return grid_unknown(g, i); }

// ---------------------------------------------------------------------------
template <typename T>
__global__ void masked_stat_kernel(Grid g, const T* x, int what, double* out, double* partials,
                                   unsigned int* counter, EpsParams ep, EpsSlot* slot, double* norm_out) {
    __shared__ double sm[32];
    double acc = 0.0;
    // unconditional loads (in bounds for every i), masked afterwards, so that
    // the unrolled iterations keep several loads in flight
#pragma unroll 4
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.size;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        const double t = (what == 0) ? fabs(v) : v * v;
        if (grid_inner(g, i)) acc += t;
    }
    double bs = block_sum(acc, sm);
    double tot = 0.0;
    if (grid_sum_last(bs, partials, counter, &tot, sm) && threadIdx.x == 0) {
        double r = (what == 0) ? tot : sqrt(tot);
        if (out) *out = r;
        if (norm_out) *norm_out = r;
        if (slot) set_eps_slot(slot, ep, r, ep.unit != 0, nullptr);
    }
}

// Scalar grids (nc = 1): the interior is (n-1)^(d-1) rows of n-1 contiguous
// entries.  One warp per row, lanes along x, rows dealt to warps in a fixed
// order (reproducible sums); one integer division per row instead of two per
// entry, and one floating-point operation per entry.  FP32 vectors are summed
// in FP32 within a row, then in FP64.  (The FP64 pipe runs at 1/64 of the
// FP32 rate on this GPU: converting every entry to FP64, or FP64 compares and
// predicated-off FP64 instructions of an unrolled loop, made these reductions
// bound by that pipe.)
constexpr int kRowWarps = kVecThreads / 32;

__host__ __device__ __forceinline__ long long interior_rows(const Grid& g) {
    const long long m = g.n - 1;
    return g.d == 3 ? m * m : m;
}

// Offset of the first entry (x = 0) of interior row r.
__device__ __forceinline__ long long interior_row_base(const Grid& g, unsigned int r) {
    const unsigned int m = (unsigned int)(g.n - 1);
    if (g.d == 2) return (long long)(r + 1) * g.sy;
    const unsigned int zz = r / m, yy = r - zz * m;
    return (long long)(zz + 1) * g.sz + (long long)(yy + 1) * g.sy;
}

// |v| without a floating-point instruction (the FP64 pipe is the scarce one)
__device__ __forceinline__ double abs_bits(double v) {
    return __longlong_as_double(__double_as_longlong(v) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float abs_bits(float v) { return __int_as_float(__float_as_int(v) & 0x7fffffff); }

// Sum over the interior entries x = 1 .. nx-2 of one row taken by lane `lane`
// (every 32nd entry): |v| (WHAT = 0) or v^2 (WHAT = 1).  Exactly one
// floating-point operation per entry; FP32 rows are summed in FP32 (at most
// 16 entries a lane up to n = 512), then added in FP64.
template <typename T, int WHAT>
__device__ __forceinline__ double row_stat(const T* __restrict__ row, int nx, int lane) {
    T f = T(0);
#pragma unroll 4
    for (int x = 1 + lane; x < nx - 1; x += 32) {
        const T v = row[x];
        if (WHAT == 0)
            f += abs_bits(v);
        else
            f = fma(v, v, f);
    }
    return (double)f;
}

template <typename T, int WHAT>
__global__ void __launch_bounds__(kVecThreads) masked_stat_rows_kernel(Grid g, const T* __restrict__ x, double* out,
                                                                       double* partials, unsigned int* counter,
                                                                       EpsParams ep, EpsSlot* slot,
                                                                       double* norm_out) {
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31;
    const unsigned int nrows = (unsigned int)interior_rows(g);
    const unsigned int wstride = gridDim.x * kRowWarps;
    double acc = 0.0;
    for (unsigned int r = blockIdx.x * kRowWarps + (threadIdx.x >> 5); r < nrows; r += wstride)
        acc += row_stat<T, WHAT>(x + JFNK_IDX(interior_row_base(g, r), g.size - g.nx + 1), g.nx, lane);
    double bs = block_sum(acc, sm);
    double tot = 0.0;
    if (grid_sum_last(bs, partials, counter, &tot, sm) && threadIdx.x == 0) {
        double res = (WHAT == 0) ? tot : sqrt(tot);
        if (out) *out = res;
        if (norm_out) *norm_out = res;
        if (slot) set_eps_slot(slot, ep, res, ep.unit != 0, nullptr);
    }
}

// at most kVecBlocks blocks (8 per SM); up to 2048 blocks, one row a warp at
// 129^3, measured slower (30 against 24 us for two FP32 norms at 129^3)
static int row_blocks(long long rows) {
    long long b = (rows + kRowWarps - 1) / kRowWarps;
    return (int)(b < kVecBlocks ? (b < 1 ? 1 : b) : kVecBlocks);
}

template <typename T>
static jfnk_status launch_masked_stat(const Grid& g, const T* x, int what, double* out, const EpsParams& ep,
                                      EpsSlot* slot, double* norm_out, RedScratch* red, cudaStream_t st) {
    if (g.nc == 1 && !g.beam && g.n >= 2 && g.size <= 0x7fffffffLL) {
        const int nb = row_blocks(interior_rows(g));
        if (what == 0)
            masked_stat_rows_kernel<T, 0><<<nb, kVecThreads, 0, st>>>(g, x, out, red->partial, &red->counter[0], ep,
                                                                      slot, norm_out);
        else
            masked_stat_rows_kernel<T, 1><<<nb, kVecThreads, 0, st>>>(g, x, out, red->partial, &red->counter[0], ep,
                                                                      slot, norm_out);
    } else {
        masked_stat_kernel<T><<<vec_blocks(g.size), kVecThreads, 0, st>>>(g, x, what, out, red->partial,
                                                                          &red->counter[0], ep, slot, norm_out);
    }
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T>
jfnk_status masked_stat(const Grid& g, const T* x, int what, double* out, RedScratch* red, cudaStream_t st) {
    EpsParams ep{};
    return launch_masked_stat<T>(g, x, what, out, ep, nullptr, nullptr, red, st);
}

template <typename T>
jfnk_status norm_to_eps(const Grid& g, const T* v, const EpsParams& ep, EpsSlot* slot, double* norm_out,
                        RedScratch* red, cudaStream_t st) {
    return launch_masked_stat<T>(g, v, 1, nullptr, ep, slot, norm_out, red, st);
}

template jfnk_status masked_stat<float>(const Grid&, const float*, int, double*, RedScratch*, cudaStream_t);
template jfnk_status masked_stat<double>(const Grid&, const double*, int, double*, RedScratch*, cudaStream_t);
template jfnk_status norm_to_eps<float>(const Grid&, const float*, const EpsParams&, EpsSlot*, double*,
                                        RedScratch*, cudaStream_t);
template jfnk_status norm_to_eps<double>(const Grid&, const double*, const EpsParams&, EpsSlot*, double*,
                                         RedScratch*, cudaStream_t);

// ---------------------------------------------------------------------------
// multi-dot: blockIdx.y selects a group of 8 vectors
constexpr int kDotGroup = 8;

template <int NG>
__device__ __forceinline__ void dot_group(const double* __restrict__ w, const double* __restrict__ V, long long ld,
                                          long long len, double* acc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < NG; ++k) acc[k] = fma(wi, V[(long long)k * ld + i], acc[k]);
    }
}
__global__ void multi_dot_kernel(const double* __restrict__ w, const double* __restrict__ V, long long ld,
                                 long long len, int m, double* h, double* partials, unsigned int* counter) {
    __shared__ double sm[kDotGroup][32];
    __shared__ int s_last;
    const int g0 = blockIdx.y * kDotGroup;
    const int ng = min(kDotGroup, m - g0);
    double acc[kDotGroup];
#pragma unroll
    for (int k = 0; k < kDotGroup; ++k) acc[k] = 0.0;
    // exactly ng FP64 FMAs per entry (a loop unrolled to kDotGroup with the
    // surplus predicated off still spends FP64-pipe issue on them)
    switch (ng) {
        case 1: dot_group<1>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 2: dot_group<2>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 3: dot_group<3>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 4: dot_group<4>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 5: dot_group<5>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 6: dot_group<6>(w, V + (long long)g0 * ld, ld, len, acc); break;
        case 7: dot_group<7>(w, V + (long long)g0 * ld, ld, len, acc); break;
        default: dot_group<8>(w, V + (long long)g0 * ld, ld, len, acc); break;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDotGroup; ++k) {
        double v = warp_sum(acc[k]);
        if (lane == 0) sm[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDotGroup && threadIdx.x < ng) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sm[threadIdx.x][q];
        partials[(long long)(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int nb = gridDim.x * gridDim.y;
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: each warp sums one vector's partials in order
    for (int k = wid; k < m; k += blockDim.x >> 5) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&partials[(long long)k * gridDim.x + b]);
        s = warp_sum(s);
        if (lane == 0) h[k] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

jfnk_status multi_dot(const double* w, const double* V, long long ld, long long len, int m, double* h,
                      double* partials, unsigned int* counter, cudaStream_t st) {
    if (m <= 0) return JFNK_OK;
    int gx = vec_blocks(len);
    if (gx > kDotBlocks) gx = kDotBlocks;
    dim3 grid(gx, (m + kDotGroup - 1) / kDotGroup);
    multi_dot_kernel<<<grid, kVecThreads, 0, st>>>(w, V, ld, len, m, h, partials, counter);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

__global__ void multi_axpy_sub_kernel(double* __restrict__ w, const double* __restrict__ V, long long ld,
                                      long long len, int m, const double* __restrict__ h) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int k = 0; k < m; ++k) acc -= h[k] * V[(long long)k * ld + i];
        w[i] = acc;
    }
}

jfnk_status multi_axpy_sub(double* w, const double* V, long long ld, long long len, int m, const double* h,
                           cudaStream_t st) {
    if (m <= 0) return JFNK_OK;
    multi_axpy_sub_kernel<<<vec_blocks(len), kVecThreads, 0, st>>>(w, V, ld, len, m, h);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

__global__ void sumsq_kernel(const double* __restrict__ w, long long len, double* nrm_out, double* partials,
                             unsigned int* counter) {
    __shared__ double sm[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        double v = w[i];
        acc += v * v;
    }
    double bs = block_sum(acc, sm);
    double tot = 0.0;
    if (grid_sum_last(bs, partials, counter, &tot, sm) && threadIdx.x == 0) *nrm_out = sqrt(tot);
}

__global__ void scale_inv_kernel(double* __restrict__ y, const double* __restrict__ x, long long len,
                                 const double* nrm) {
    const double n = *nrm;
    const double s = n > 0.0 ? 1.0 / n : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

jfnk_status normalize(double* w, long long len, double* nrm_out, double* partials, unsigned int* counter,
                      cudaStream_t st) {
    sumsq_kernel<<<vec_blocks(len), kVecThreads, 0, st>>>(w, len, nrm_out, partials, counter);
    JFNK_LAUNCH_CHECK();
    scale_inv_kernel<<<vec_blocks(len), kVecThreads, 0, st>>>(w, w, len, nrm_out);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

jfnk_status scale_by_inv(double* y, const double* x, long long len, const double* nrm, cudaStream_t st) {
    scale_inv_kernel<<<vec_blocks(len), kVecThreads, 0, st>>>(y, x, len, nrm);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

// ---------------------------------------------------------------------------
template <typename TZ>
__global__ void combine_kernel(double* __restrict__ x, const TZ* __restrict__ Z, long long ld, long long len,
                               int m, const double* __restrict__ c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        double acc = x[i];
        for (int k = 0; k < m; ++k) acc += c[k] * (double)Z[(long long)k * ld + i];
        x[i] = acc;
    }
}

template <typename TZ>
jfnk_status combine(double* x, const TZ* Z, long long ld, long long len, int m, const double* c, cudaStream_t st) {
    if (m <= 0) return JFNK_OK;
    combine_kernel<TZ><<<vec_blocks(len), kVecThreads, 0, st>>>(x, Z, ld, len, m, c);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status combine<float>(double*, const float*, long long, long long, int, const double*, cudaStream_t);
template jfnk_status combine<double>(double*, const double*, long long, long long, int, const double*, cudaStream_t);

template <typename T>
__global__ void axpby_kernel(T* __restrict__ y, const T* __restrict__ x, T a, T b, long long len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

template <typename T>
jfnk_status axpby(T* y, const T* x, double a, double b, long long len, cudaStream_t st) {
    axpby_kernel<T><<<vec_blocks(len), kVecThreads, 0, st>>>(y, x, (T)a, (T)b, len);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status axpby<float>(float*, const float*, double, double, long long, cudaStream_t);
template jfnk_status axpby<double>(double*, const double*, double, double, long long, cudaStream_t);

__global__ void add_scaled_kernel(double* __restrict__ z, const double* __restrict__ x, double a,
                                  const double* __restrict__ y, long long len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        z[i] = x[i] + a * y[i];
}

jfnk_status add_scaled(double* z, const double* x, double a, const double* y, long long len, cudaStream_t st) {
    add_scaled_kernel<<<vec_blocks(len), kVecThreads, 0, st>>>(z, x, a, y, len);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename TO, typename TI>
__global__ void cast_kernel(TO* __restrict__ y, const TI* __restrict__ x, long long len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (TO)x[i];
}

template <typename TO, typename TI>
jfnk_status cast_copy(TO* y, const TI* x, long long len, cudaStream_t st) {
    cast_kernel<TO, TI><<<vec_blocks(len), kVecThreads, 0, st>>>(y, x, len);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status cast_copy<float, double>(float*, const double*, long long, cudaStream_t);
template jfnk_status cast_copy<double, float>(double*, const float*, long long, cudaStream_t);
template jfnk_status cast_copy<double, double>(double*, const double*, long long, cudaStream_t);
template jfnk_status cast_copy<float, float>(float*, const float*, long long, cudaStream_t);

template <typename TO, typename TI>
__global__ void cast_scale_interior_kernel(TO* __restrict__ y, const TI* __restrict__ x, double a, Grid g) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.size;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = grid_inner(g, i) ? (TO)(a * (double)x[i]) : TO(0);
}

template <typename TO, typename TI>
jfnk_status cast_scale_interior(TO* y, const TI* x, double a, const Grid& g, cudaStream_t st) {
    cast_scale_interior_kernel<TO, TI><<<vec_blocks(g.size), kVecThreads, 0, st>>>(y, x, a, g);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status cast_scale_interior<float, double>(float*, const double*, double, const Grid&, cudaStream_t);
template jfnk_status cast_scale_interior<double, double>(double*, const double*, double, const Grid&, cudaStream_t);
template jfnk_status cast_scale_interior<double, float>(double*, const float*, double, const Grid&, cudaStream_t);
template jfnk_status cast_scale_interior<float, float>(float*, const float*, double, const Grid&, cudaStream_t);

template <typename T>
__global__ void add_inplace_kernel(T* __restrict__ s, const T* __restrict__ d, long long len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        s[i] += d[i];
}

template <typename T>
jfnk_status add_inplace(T* s, const T* d, long long len, cudaStream_t st) {
    add_inplace_kernel<T><<<vec_blocks(len), kVecThreads, 0, st>>>(s, d, len);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status add_inplace<float>(float*, const float*, long long, cudaStream_t);
template jfnk_status add_inplace<double>(double*, const double*, long long, cudaStream_t);

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): state advances by GAMMA, output is the
// 64-bit finaliser of the state.  Counter form: output c of stream k is
// finaliser(k + (c+1) GAMMA).
__device__ __forceinline__ uint64_t splitmix_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void splitmix_kernel(Grid g, T* v, uint64_t key) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.size;
         i += (long long)gridDim.x * blockDim.x) {
        T val = T(0);
        if (grid_inner(g, i)) {
            uint64_t z = splitmix_finalise(key + ((uint64_t)i + 1ULL) * 0x9E3779B97F4A7C15ULL);
            double u = (double)(z >> 11) * 0x1.0p-53;
            val = (T)(u * 2.0 - 1.0);
        }
        v[i] = val;
    }
}

template <typename T>
jfnk_status splitmix_start(const Grid& g, T* v, uint64_t seed, int level, cudaStream_t st) {
    const uint64_t key = seed + (uint64_t)level * 0xD1B54A32D192ED03ULL;
    splitmix_kernel<T><<<vec_blocks(g.size), kVecThreads, 0, st>>>(g, v, key);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status splitmix_start<float>(const Grid&, float*, uint64_t, int, cudaStream_t);
template jfnk_status splitmix_start<double>(const Grid&, double*, uint64_t, int, cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void cheb_table_kernel(const double* lam, double lo, double hi, int degree, ChebTable* t, int* status) {
    const double l = *lam;
    if (!(l > 0.0) || !isfinite(l)) {
        if (status) atomicOr(status, 2);
    }
    double theta, c1, c2;
    cheb_coeffs(l, lo, hi, 0, theta, c1, c2);
    t->theta_inv = 1.0 / theta;
    t->theta_invf = (float)(1.0 / theta);
    for (int i = 0; i < degree && i < kMaxChebDegree; ++i) {
        cheb_coeffs(l, lo, hi, i, theta, c1, c2);
        t->c1[i] = c1;
        t->c2[i] = c2;
        t->c1f[i] = (float)c1;
        t->c2f[i] = (float)c2;
    }
}

jfnk_status cheb_table(const double* lam, double lo, double hi, int degree, ChebTable* t, int* status,
                       cudaStream_t st) {
    cheb_table_kernel<<<1, 1, 0, st>>>(lam, lo, hi, degree, t, status);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

__global__ void copy_scalar_kernel(double* d, const double* s) { *d = *s; }
jfnk_status copy_scalar(double* dst, const double* src, cudaStream_t st) {
    copy_scalar_kernel<<<1, 1, 0, st>>>(dst, src);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

}  // namespace jfnk

namespace jfnk {

template <typename T>
__global__ void cheb_start_zero_kernel(Grid g, const T* __restrict__ b, T* __restrict__ r, T* __restrict__ d,
                                       const ChebTable* cheb, EpsParams ep, EpsSlot* slot, double* partials,
                                       unsigned int* counter) {
    __shared__ double sm[32];
    const double ti = cheb->theta_inv;
    double acc = 0.0;
#pragma unroll 4
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.size;
         i += (long long)gridDim.x * blockDim.x) {
        const bool in = grid_inner(g, i);
        T bv = b[i];  // loaded unconditionally (see masked_stat_kernel)
        if (!in) bv = T(0);
        const T dv = (T)((double)bv * ti);
        r[i] = bv;
        d[i] = dv;
        acc += (double)dv * (double)dv;
    }
    double bs = block_sum(acc, sm);
    double tot = 0.0;
    if (grid_sum_last(bs, partials, counter, &tot, sm) && threadIdx.x == 0) {
        double e = eps_formula(ep.mode, ep.n_unknowns, *ep.xstat, sqrt(tot));
        double inv = e > 0.0 ? 1.0 / e : 0.0;
        slot->e = e;
        slot->inv = inv;
        slot->ef = (float)e;
        slot->invf = (float)inv;
    }
}

// The same over the rows of a scalar grid (every row, so that the boundary
// entries of r and d are written as zeros): one warp per row, the interior
// test per row and per x, FP32 arithmetic for FP32 vectors (d = b / theta in
// the vector's precision, the norm summed as in masked_stat_rows_kernel).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cheb_start_zero_rows_kernel(
    Grid g, const T* __restrict__ b, T* __restrict__ r, T* __restrict__ d, const ChebTable* cheb, EpsParams ep,
    EpsSlot* slot, double* partials, unsigned int* counter) {
    __shared__ double sm[32];
    const T ti = sizeof(T) == 4 ? (T)cheb->theta_invf : (T)cheb->theta_inv;
    const int lane = threadIdx.x & 31;
    const unsigned int nrows = (unsigned int)(g.ny * g.nz);
    const unsigned int wstride = gridDim.x * kRowWarps;
    const int nx = g.nx;
    double acc = 0.0;
    for (unsigned int row = blockIdx.x * kRowWarps + (threadIdx.x >> 5); row < nrows; row += wstride) {
        const unsigned int zz = row / (unsigned int)g.ny, yy = row - zz * (unsigned int)g.ny;
        const bool inner_row = yy > 0 && yy < (unsigned int)g.ny - 1 && (g.d == 2 || (zz > 0 && zz < (unsigned int)g.nz - 1));
        const long long base = JFNK_IDX((long long)row * g.sy, g.size - g.nx + 1);
        const T* br = b + base;
        T* rr = r + base;
        T* dr = d + base;
        T f = T(0);
#pragma unroll 4
        for (int x = lane; x < nx; x += 32) {
            const bool in = inner_row && x > 0 && x < nx - 1;
            const T bv = in ? br[x] : T(0);
            const T dv = bv * ti;
            rr[x] = bv;
            dr[x] = dv;
            f = fma(dv, dv, f);
        }
        acc += (double)f;
    }
    double bs = block_sum(acc, sm);
    double tot = 0.0;
    if (grid_sum_last(bs, partials, counter, &tot, sm) && threadIdx.x == 0) {
        double e = eps_formula(ep.mode, ep.n_unknowns, *ep.xstat, sqrt(tot));
        double inv = e > 0.0 ? 1.0 / e : 0.0;
        slot->e = e;
        slot->inv = inv;
        slot->ef = (float)e;
        slot->invf = (float)inv;
    }
}

template <typename T>
jfnk_status cheb_start_zero(const Grid& g, const T* b, T* r, T* d, const ChebTable* cheb, const EpsParams& ep,
                            EpsSlot* slot, RedScratch* red, cudaStream_t st) {
    if (g.nc == 1 && !g.beam && g.n >= 2 && g.size <= 0x7fffffffLL) {
        cheb_start_zero_rows_kernel<T><<<row_blocks((long long)g.ny * g.nz), kVecThreads, 0, st>>>(
            g, b, r, d, cheb, ep, slot, red->partial, &red->counter[0]);
    } else {
        cheb_start_zero_kernel<T><<<vec_blocks(g.size), kVecThreads, 0, st>>>(g, b, r, d, cheb, ep, slot,
                                                                              red->partial, &red->counter[0]);
    }
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status cheb_start_zero<float>(const Grid&, const float*, float*, float*, const ChebTable*,
                                            const EpsParams&, EpsSlot*, RedScratch*, cudaStream_t);
template jfnk_status cheb_start_zero<double>(const Grid&, const double*, double*, double*, const ChebTable*,
                                             const EpsParams&, EpsSlot*, RedScratch*, cudaStream_t);

template <typename T>
__global__ void scale_inplace_inv_kernel(T* v, long long len, const double* nrm) {
    const double n = *nrm;
    const T s = (T)(n > 0.0 ? 1.0 / n : 0.0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        v[i] *= s;
}

template <typename T>
jfnk_status scale_inplace_inv(T* v, long long len, const double* nrm, cudaStream_t st) {
    scale_inplace_inv_kernel<T><<<vec_blocks(len), kVecThreads, 0, st>>>(v, len, nrm);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status scale_inplace_inv<float>(float*, long long, const double*, cudaStream_t);
template jfnk_status scale_inplace_inv<double>(double*, long long, const double*, cudaStream_t);

__global__ void set_eps_kernel(EpsSlot* s, double e) {
    double inv = e > 0.0 ? 1.0 / e : 0.0;
    s->e = e;
    s->inv = inv;
    s->ef = (float)e;
    s->invf = (float)inv;
}
jfnk_status set_eps(EpsSlot* slot, double e, cudaStream_t st) {
    set_eps_kernel<<<1, 1, 0, st>>>(slot, e);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

__global__ void ratio_kernel(double* lam, const double* a, const double* b) {
    const double bb = *b;
    *lam = bb > 0.0 ? *a / bb : 0.0;
}
jfnk_status ratio_scalar(double* lam, const double* a, const double* b, cudaStream_t st) {
    ratio_kernel<<<1, 1, 0, st>>>(lam, a, b);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

}  // namespace jfnk
