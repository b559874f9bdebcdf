// Vector kernels: reductions, BLAS-1, casts, start vectors.
#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

// Interior-masked reductions over a node grid.  what: 0 sum|x|, 1 sum x^2.
// Result: *out = sum|x| or sqrt(sum x^2) (deterministic).
template <typename T>
jfnk_status masked_stat(const Grid& g, const T* x, int what, double* out, RedScratch* red, cudaStream_t st);

// ||v||_2 over interior nodes, then the FD step of v into *slot (Sec. 1 formula).
template <typename T>
jfnk_status norm_to_eps(const Grid& g, const T* v, const EpsParams& ep, EpsSlot* slot, double* norm_out,
                        RedScratch* red, cudaStream_t st);

// h[i] = <w, V_i> for i < m, V_i = V + i * ld (flat dot over all entries;
// boundary entries of Krylov vectors are zero).  partials: >= m * kDotBlocks.
constexpr int kDotBlocks = 304;
jfnk_status multi_dot(const double* w, const double* V, long long ld, long long len, int m, double* h,
                      double* partials, unsigned int* counter, cudaStream_t st);
// w -= sum_i h[i] V_i  (h on device)
jfnk_status multi_axpy_sub(double* w, const double* V, long long ld, long long len, int m, const double* h,
                           cudaStream_t st);
// nrm = ||w||, w *= 1/nrm (two kernels); writes *nrm_out (device)
jfnk_status normalize(double* w, long long len, double* nrm_out, double* partials, unsigned int* counter,
                      cudaStream_t st);
// y = x * (1/nrm) with nrm a device scalar (0 -> y = 0)
jfnk_status scale_by_inv(double* y, const double* x, long long len, const double* nrm, cudaStream_t st);

// x += sum_i c[i] Z_i with c on device, Z in TZ (float or double)
template <typename TZ>
jfnk_status combine(double* x, const TZ* Z, long long ld, long long len, int m, const double* c, cudaStream_t st);

// y = a x + b y (host scalars), y, x of the same type
template <typename T>
jfnk_status axpby(T* y, const T* x, double a, double b, long long len, cudaStream_t st);
// z = x + a y
jfnk_status add_scaled(double* z, const double* x, double a, const double* y, long long len, cudaStream_t st);
// y = (TO) x
template <typename TO, typename TI>
jfnk_status cast_copy(TO* y, const TI* x, long long len, cudaStream_t st);
// y = (TO)(a x) with x on interior nodes only, boundary 0
template <typename TO, typename TI>
jfnk_status cast_scale_interior(TO* y, const TI* x, double a, const Grid& g, cudaStream_t st);
// s += d
template <typename T>
jfnk_status add_inplace(T* s, const T* d, long long len, cudaStream_t st);

// SplitMix64 start vector of the power method: uniform [-1,1) on interior nodes
// from stream key seed + level * 0xD1B54A32D192ED03, counter = node index.
template <typename T>
jfnk_status splitmix_start(const Grid& g, T* v, uint64_t seed, int level, cudaStream_t st);

// Chebyshev table for the level from lambda (device), interval [lo, hi]*lambda
jfnk_status cheb_table(const double* lam, double lo, double hi, int degree, ChebTable* t, int* status,
                       cudaStream_t st);
// Power-method step on device: lam = nrm; status if not finite.
jfnk_status copy_scalar(double* dst, const double* src, cudaStream_t st);

}  // namespace jfnk

namespace jfnk {
// Chebyshev start from s = 0: r = b, d = b / theta, ||d|| -> FD step of d
template <typename T>
jfnk_status cheb_start_zero(const Grid& g, const T* b, T* r, T* d, const ChebTable* cheb, const EpsParams& ep,
                            EpsSlot* slot, RedScratch* red, cudaStream_t st);
// v *= 1/nrm (device scalar), any precision
template <typename T>
jfnk_status scale_inplace_inv(T* v, long long len, const double* nrm, cudaStream_t st);
// set an FD-step slot from the host value e
jfnk_status set_eps(EpsSlot* slot, double e, cudaStream_t st);
// lam = a / b (device scalars)
jfnk_status ratio_scalar(double* lam, const double* a, const double* b, cudaStream_t st);
}  // namespace jfnk
