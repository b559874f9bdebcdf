// Hyperelastic beam (Sec. 3): element kernels and transfers.
#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

// scratch entries of the beam element kernels: 24 per element
inline long long beam_scratch_count(const Grid& g) { return g.beam ? 24LL * g.elements() : 0; }

// Mode as for launch_stencil; a.lh carries 1/h, a.node_scale is unused (1).
template <typename T>
jfnk_status launch_beam(Mode mode, const StencilArgs<T>& a, cudaStream_t st);

// c = R f (projection = false) or the projection of the iterate (true)
template <typename T>
jfnk_status beam_restrict(const Grid& gf, const Grid& gc, const T* f, T* c, bool projection, cudaStream_t st);
// s += I c
template <typename T>
jfnk_status beam_prolong_add(const Grid& gc, const Grid& gf, const T* c, T* s, cudaStream_t st);

}  // namespace jfnk
