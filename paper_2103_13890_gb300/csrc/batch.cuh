// Batched kernels: one launch applies a level operation to every active
// instance of a batch of independent problems of uneven sizes.  Each CTA
// reads a work item (instance, tile or block) and that instance's operands
// from descriptor arrays in device memory; reductions complete per instance
// (each instance's CTAs form one segment of the last-block reduction).
#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

// 2D row-segment tile of one instance
struct BTile {
    int inst;
    int x0, y0, y1, txo;
    int bid, nblk;  // index among the instance's CTAs, their count
    int pad;
};

// work item of a batched vector operation
struct BItem {
    int inst, bid, nblk, pad;
};

// per-instance operands of a batched vector operation
struct BVec {
    Grid g;            // grid of x / y
    Grid gc;           // coarse grid (transfers)
    void* y;           // output
    const void* x;     // input
    const void* x2;    // second input
    void* y2;          // second output
    double a, b;       // scalars
    const double* dsc; // device scalar operand
    double* out;       // reduction result(s)
    EpsSlot* slot;     // FD step produced by a norm
    EpsParams ep;
    const ChebTable* cheb;
    double* partials;  // this instance's reduction scratch
    unsigned int* counter;
    long long ld;      // leading dimension of a vector block (FGMRES bases)
    int m;             // number of vectors in a block operation
    int what;          // op detail (statistic kind, projection flag, ...)
    uint64_t key;      // SplitMix64 stream key
};

enum class BOp : int {
    CAST_D2T = 0,    // y(T) = x(double)
    CAST_T2D = 1,    // y(double) = x(T)
    COPY_T = 2,      // y = x
    AXPBY_D = 3,     // y = a x + b y              (double)
    ADDSC_D = 4,     // y = x + a x2              (double)
    SCALE_INV_T = 5, // y = x / *dsc (0 if *dsc == 0)
    STAT = 6,        // out = sum|x| (what 0) or ||x|| (what 1), interior; slot (if set) = FD step
    CHEB_START = 7,  // y = r = b(x) interior, y2 = d = b / theta, s(x2 as output) = 0; ||d|| -> slot
    RESTRICT = 8,    // y(gc) = I^T x (what 1: projection 2^-d, boundary injection)
    PROLONG_ADD = 9, // y += I x(gc)
    SPLITMIX = 10,   // y = uniform [-1,1) start vector from key (interior)
    MDOT = 11,       // out[k] = <x, x2 + k ld>, k < m   (double)
    MAXPY_SUB = 12,  // y -= sum_k out[k] (x2 + k ld)   (double; out read as coefficients)
    COMBINE_T = 13,  // y(double) += sum_k dsc[k] (x(T) + k ld)
    CAST_SCALE_INT_D = 14,  // y(double) = a x(double) on interior, 0 on the boundary
};

// Tiny per-instance scalar kernels (one thread per instance)
enum class BScalar : int {
    RATIO = 0,       // *out = *x / *x2    (lambda = ||Jv|| / ||v||)
    CHEB_TABLE = 1,  // cheb table from *x with [a, b] and degree m
    SET_EPS = 2,     // slot from a
};
struct BScal {
    double* out;
    const double* x;
    const double* x2;
    double a, b;
    int m;
    ChebTable* cheb;
    EpsSlot* slot;
    int* status;
};

// grid > 0 (< ntiles): persistent launch of `grid` CTAs looping over the tiles
template <typename T>
jfnk_status launch_stencil2d_batched(Mode mode, const StencilArgs<T>* dev_args, const BTile* dev_tiles, int ntiles,
                                     int bx, cudaStream_t st, int grid = 0);

template <typename T>
jfnk_status launch_bvec(BOp op, const BVec* dev_desc, const BItem* dev_items, int nitems, cudaStream_t st);

jfnk_status launch_bscalar(BScalar op, const BScal* dev_desc, int count, cudaStream_t st);

}  // namespace jfnk
