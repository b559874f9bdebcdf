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

// Layout of the z-marching kernels' scratch (stencil_ep.cu): Cz[4][n+1][n][n],
// per plane and element column the column's parts of its 4 nodes in the plane.
__host__ __device__ inline long long zm3d_plane_stride(int n) { return (long long)(n + 1) * n * n; }
__host__ __device__ inline long long zm3d_scratch_count(int n) { return 4 * zm3d_plane_stride(n); }

// Scratch entries for grid g with one element a thread (zm = false) or with
// the z-marching element columns (zm = true).
inline long long ep3d_scratch_need(const Grid& g, bool zm) {
    return g.d == 3 ? (zm ? zm3d_scratch_count(g.n) : ep3d_scratch_count(g)) : 0;
}

// True when the element-parallel kernels run for these arguments: levels with
// n <= ep_max_n, and levels with n >= zm_min_n (> 0), which march element
// columns along z (the adjoint keeps one element a thread and follows
// ep_max_n only).
template <typename T>
inline bool ep3d_use(const StencilArgs<T>& a, bool adj = false) {
    const bool zm = !adj && a.zm_min_n > 0 && a.g.n >= a.zm_min_n;
    return a.face != nullptr && a.g.d == 3 && !a.g.beam && (a.g.n <= a.ep_max_n || zm) &&
           ep3d_scratch_need(a.g, zm) <= a.face_cap;
}

// Sets the cluster kernels' attributes on the current device (once) and
// returns whether a cluster of their largest size fits there.  Called by the
// launcher; callers that capture launches into a graph call it first.
bool ep3d_cluster_init();

// adj: the vector-Jacobian product (J^T v, and (dF/dkappa)^T v into a.dkout)
// in place of the FD action.
template <typename T>
jfnk_status launch_ep3d(Prob prob, Mode mode, bool adj, const StencilArgs<T>& a, cudaStream_t st);

}  // namespace jfnk
