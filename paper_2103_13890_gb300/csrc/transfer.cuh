#pragma once
#include "common.cuh"

namespace jfnk {

// projection=false: c = R f = I^T f (coarse boundary 0)
// projection=true:  c = P f = 2^-d I^T f on interior coarse nodes, injection on the boundary
template <typename T>
jfnk_status restrict_to(const Grid& gf, const Grid& gc, const T* f, T* c, bool projection, cudaStream_t st);
// s += I c
template <typename T>
jfnk_status prolong_add(const Grid& gc, const Grid& gf, const T* c, T* s, cudaStream_t st);
jfnk_status coarsen_kappa(int nc, const double* kf, double* kc, cudaStream_t st);
// tab_dev: three tables of nx doubles (I1, I3, Ic), see transfer.cu
jfnk_status mms_load(const Grid& g, const double* tab_dev, double* b, cudaStream_t st);

}  // namespace jfnk
