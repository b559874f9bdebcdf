// Internal definitions shared by the libjfnk.so translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "jfnk.h"

namespace jfnk {

// Structured node grid of one level: n elements per direction, full node grid
// including Dirichlet boundary nodes, x fastest, densely packed.
struct Grid {
    int d;             // 2 or 3
    int n;             // elements per direction
    int nx, ny, nz;    // nodes per direction (nz = 1 in 2D)
    long long sy, sz;  // strides of y and z in elements
    long long size;    // number of entries

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
        return g;
    }
    long long interior() const {
        long long m = (long long)(n - 1) * (n - 1);
        return d == 3 ? m * (n - 1) : m;
    }
};

// Error reporting (thread-local message, see jfnk_last_error)
void set_error(const char* fmt, ...);
void count_launch(int k = 1);

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
