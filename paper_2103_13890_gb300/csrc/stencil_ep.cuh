// Element-parallel 3D element-residual kernels (two launches, no halo, no
// barrier inside the element phase; FP32 levels with at most 512 elements run
// both phases in one CTA).
#pragma once
#include "stencil.cuh"

namespace jfnk {

// Scratch entries the element-parallel kernels need for grid g: 8 per element.
inline long long ep3d_scratch_count(const Grid& g) {
    return g.d == 3 ? 8LL * g.n * g.n * g.n : 0;
}

// True when the element-parallel kernels run for these arguments.
template <typename T>
inline bool ep3d_use(const StencilArgs<T>& a) {
    return a.face != nullptr && a.g.d == 3 && !a.g.beam && a.g.n <= a.ep_max_n &&
           ep3d_scratch_count(a.g) <= a.face_cap;
}

// adj: the vector-Jacobian product (J^T v, and (dF/dkappa)^T v into a.dkout)
// in place of the FD action.
template <typename T>
jfnk_status launch_ep3d(Prob prob, Mode mode, bool adj, const StencilArgs<T>& a, cudaStream_t st);

}  // namespace jfnk
