#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

constexpr int kV2Threads = 1024;  // at most n x BY threads per CTA
constexpr int kV3Threads = 512;   // (n/2) x BY threads of the FP32 paired-element variant

// Tiling of the halo-free 3D kernel and the layout of its face buffer.
struct V2Geom {
    int n;    // elements per direction (multiple of 32)
    int BY;   // element rows per CTA (the largest divisor of n with n BY <= the thread cap)
    int Ty;   // y tiles (n / BY)
    int Tz;   // z chunks
    int ZC;   // layers per chunk (last one may be shorter)
    long long ylo, yhi, zlo, zhi;  // offsets of the four face arrays
    long long face_count;          // total entries
};

bool v2_applicable(const Grid& g);
// max_threads: cap on n x BY (<= kV2Threads); CTAs of that size share an SM
// kV2Threads / (n BY) at a time, which the z-chunk choice accounts for
V2Geom v2_geometry(const Grid& g, int num_sms, int max_threads = kV2Threads);
long long v2_face_count(const Grid& g, int max_threads = kV2Threads);  // 0 if the v2 kernel does not apply

template <typename T>
jfnk_status launch_stencil_v2(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st);
// FP32 only: the same tiling and face fixup, two elements per thread in packed f32x2 arithmetic
jfnk_status launch_stencil_v3(Prob prob, Mode mode, const StencilArgs<float>& a, cudaStream_t st);
// face entries of that variant with ctas_per_sm resident CTAs per SM (0 if it does not apply)
long long v3_face_count(const Grid& g, int max_threads, int ctas_per_sm);

}  // namespace jfnk
