#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

constexpr int kV2Threads = 1024;  // n x BY threads per CTA

// Tiling of the halo-free 3D kernel and the layout of its face buffer.
struct V2Geom {
    int n;    // elements per direction (multiple of 32)
    int BY;   // element rows per CTA (kV2Threads / n)
    int Ty;   // y tiles (n / BY)
    int Tz;   // z chunks
    int ZC;   // layers per chunk (last one may be shorter)
    long long ylo, yhi, zlo, zhi;  // offsets of the four face arrays
    long long face_count;          // total entries
};

bool v2_applicable(const Grid& g);
V2Geom v2_geometry(const Grid& g, int num_sms);
long long v2_face_count(const Grid& g);  // 0 if the v2 kernel does not apply

template <typename T>
jfnk_status launch_stencil_v2(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st);

}  // namespace jfnk
