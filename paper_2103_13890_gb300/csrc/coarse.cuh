#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

template <typename T>
struct CoarseArgs {
    Grid g;                // level-0 grid
    const T* x;            // x_0
    const T* Ax;           // A(x_0)
    const T* b;            // right-hand side r_0
    T* s;                  // solution (boundary 0)
    const T* kappa;        // NDK per element
    T lh;                  // Bratu lambda h^2/16
    T node_scale;          // 3h/16 (3D) or 1
    int eps_mode;          // jfnk_eps_mode
    double n_unknowns;
    const double* xstat;   // device
    double tol;
    int tol_abs;           // 1: absolute tolerance
    int maxit;
    T* V;                  // (maxit + 1) * g.size scratch
    double* H;             // (maxit + 1) * maxit scratch
    long long* iters;      // device accumulator of GMRES iterations (GE count), nullable
    int adjoint;           // 1: solve with J(x_0)^T (exact VJP) instead of the FD action
};

template <typename T>
jfnk_status launch_coarse(Prob prob, const CoarseArgs<T>& a, cudaStream_t st);
// count instances (2D Bratu, same coarse grid as a0), args in device memory
template <typename T>
jfnk_status launch_coarse_batched(const CoarseArgs<T>& a0, const CoarseArgs<T>* dev_args, int count, cudaStream_t st);

}  // namespace jfnk
