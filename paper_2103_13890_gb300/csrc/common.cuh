// Internal definitions shared by the libjfnk.so translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "jfnk.h"

namespace jfnk {

// Structured node grid of one level: n elements per direction, full node grid
// including Dirichlet boundary nodes, x fastest, densely packed.  The beam of
// the hyperelastic problem (beam = 1) has 10n x n x n elements, nc = 3
// displacement components per node (component fastest), Dirichlet data on the
// faces x = 0 and x = 10 only: its y and z faces are free, so their nodes are
// unknowns.
struct Grid {
    int d;             // 2 or 3
    int n;             // elements per direction (beam: lateral, the length has 10 n)
    int nx, ny, nz;    // nodes per direction (nz = 1 in 2D)
    long long sy, sz;  // strides of y and z in entries
    long long size;    // number of entries
    int nc;            // entries per node
    int beam;          // 1: the hyperelastic beam

    static Grid make(int d, int n) {
        Grid g;
        g.d = d;
        g.n = n;
        g.nx = n + 1;
        g.ny = n + 1;
        g.nz = (d == 3) ? n + 1 : 1;
        g.sy = g.nx;
        g.sz = (long long)g.nx * g.ny;
        g.size = g.sz * g.nz;
        g.nc = 1;
        g.beam = 0;
        return g;
    }
    static Grid make_beam(int n) {
        Grid g;
        g.d = 3;
        g.n = n;
        g.nx = 10 * n + 1;
        g.ny = n + 1;
        g.nz = n + 1;
        g.nc = 3;
        g.beam = 1;
        g.sy = (long long)g.nx * 3;
        g.sz = g.sy * g.ny;
        g.size = g.sz * g.nz;
        return g;
    }
    __host__ __device__ long long elements() const {
        if (beam) return 10LL * n * n * n;
        return d == 3 ? (long long)n * n * n : (long long)n * n;
    }
    // unknown entries (the n of the FD-step formula, Sec. 1)
    __host__ __device__ long long interior() const {
        if (beam) return (long long)(nx - 2) * ny * nz * nc;
        long long m = (long long)(n - 1) * (n - 1);
        return d == 3 ? m * (n - 1) : m;
    }
};

// Node coordinates (x, y, z) of entry i of a scalar grid (nc = 1); 32-bit
// index arithmetic where the grid allows it.
__host__ __device__ __forceinline__ void grid_coords(const Grid& g, long long i, int& x, int& y, int& z) {
    if (g.size <= 0x7fffffffLL) {
        const unsigned int ii = (unsigned int)i, sy = (unsigned int)g.sy, ny = (unsigned int)g.ny;
        const unsigned int yz = ii / sy, zz = yz / ny;
        x = (int)(ii - yz * sy);
        y = (int)(yz - zz * ny);
        z = (int)zz;
        return;
    }
    const long long yz = i / g.sy;
    x = (int)(i - yz * g.sy);
    y = (int)(yz % g.ny);
    z = (int)(yz / g.ny);
}

// True for the entries that are unknowns (not Dirichlet data) of grid g.
__host__ __device__ __forceinline__ bool grid_unknown(const Grid& g, long long i) {
    if (g.size <= 0x7fffffffLL) {  // 32-bit index arithmetic (64-bit division is a long subroutine)
        const unsigned int ii = (unsigned int)i;
        const unsigned int node = g.nc == 1 ? ii : ii / (unsigned int)g.nc;
        const unsigned int nx = (unsigned int)g.nx, ny = (unsigned int)g.ny;
        const unsigned int yz = node / nx, x = node - yz * nx;
        if (g.beam) return x > 0 && x < nx - 1;
        const unsigned int z = yz / ny, y = yz - z * ny;
        bool in = x > 0 && x < nx - 1 && y > 0 && y < ny - 1;
        if (g.d == 3) in = in && z > 0 && z < (unsigned int)g.nz - 1;
        return in;
    }
    const long long node = g.nc == 1 ? i : i / g.nc;
    const long long x = node % g.nx;
    const long long yz = node / g.nx;
    if (g.beam) return x > 0 && x < g.nx - 1;
    const long long y = yz % g.ny;
    bool in = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1;
    if (g.d == 3) {
        const long long z = yz / g.ny;
        in = in && z > 0 && z < g.nz - 1;
    }
    return in;
}

// Error reporting (thread-local message, see jfnk_last_error)
void set_error(const char* fmt, ...);
void count_launch(int k = 1);

// Bounds-checked builds (compiled with -DJFNK_DEBUG_BOUNDS): JFNK_IDX(i, n)
// checks 0 <= i < n before an access.  An index out of range is recorded (the
// source line of the first one, in a device word of its translation unit) and
// clamped into range, so the kernel neither faults nor traps and the host
// reads the record afterwards (jfnk_debug_bounds).  In normal builds the
// macro is the index itself.
typedef unsigned int (*BoundsReader)(int reset);
int register_bounds_reader(BoundsReader reader, const char* file);
#ifdef JFNK_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_line;  // one per translation unit
#ifdef __CUDACC__
__device__ __forceinline__ long long dbg_idx(long long i, long long n, unsigned int line) {
    if (i < 0 || i >= n) {
        atomicCAS(&g_bounds_line, 0u, line);
        return i < 0 ? 0 : (n > 0 ? n - 1 : 0);
    }
    return i;
}
#endif
static unsigned int read_bounds_line(int reset) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_line, sizeof(v)) != cudaSuccess) return 0xffffffffu;
    if (reset) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_bounds_line, &z, sizeof(z));
    }
    return v;
}
static const int g_bounds_registered = register_bounds_reader(&read_bounds_line, __FILE__);
#define JFNK_IDX(i, n) ::jfnk::dbg_idx((long long)(i), (long long)(n), __LINE__)
#else
#define JFNK_IDX(i, n) (i)
#endif

#define JFNK_CUDA_TRY(expr)                                                          \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::jfnk::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,            \
                              cudaGetErrorString(e_));                               \
            return JFNK_ERR_CUDA;                                                    \
        }                                                                            \
    } while (0)

#define JFNK_LAUNCH_CHECK()                                                          \
    do {                                                                             \
        ::jfnk::count_launch();                                                      \
        cudaError_t e_ = cudaGetLastError();                                         \
        if (e_ != cudaSuccess) {                                                     \
            ::jfnk::set_error("%s:%d: kernel launch: %s", __FILE__, __LINE__,        \
                              cudaGetErrorString(e_));                               \
            return JFNK_ERR_CUDA;                                                    \
        }                                                                            \
    } while (0)

#define JFNK_TRY(expr)                           \
    do {                                         \
        jfnk_status s_ = (expr);                 \
        if (s_ != JFNK_OK) return s_;            \
    } while (0)

constexpr int kNumSMs = 152;  // GB300; the launchers query the device anyway

// ---------------------------------------------------------------------------
// Device-side scalar block: all per-level scalars live in device memory so that
// a V-cycle is a fixed launch sequence (capturable in a CUDA graph).
// ---------------------------------------------------------------------------
struct LevelScalars {
    double xstat;      // sum_i |x_i| (paper eps) or ||x||_2 (fp32 eps) over interior
    double lam_max;    // power-method estimate (Sec. 2)
    double eps[4];     // FD steps of the current actions (slots)
    double nrm[4];     // norms produced by reductions (slots)
    int status;        // device-detected problems (non-finite eps, ...)
    int pad[7];
};

// Reduction scratch: per-block partial sums plus a completion counter used by
// the last-block pattern (no spinning: the last block to finish sums all
// partials in a fixed order, so results are deterministic).
constexpr int kMaxRedBlocks = 1024;
struct RedScratch {
    double partial[kMaxRedBlocks * 2];
    unsigned int counter[8];
};

}  // namespace jfnk
