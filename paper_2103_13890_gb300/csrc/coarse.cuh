#pragma once
#include "common.cuh"
#include "stencil.cuh"

namespace jfnk {

// L-BFGS preconditioner of the coarse CG (Sec. 2, "The coarse level solver"):
// kept secant pairs and the small matrices of its compact representation
// (Byrd, Nocedal & Schnabel, Math. Program. 63 (1994), Thm. 2.2):
//   H = gamma I + [S  gamma Y] [[R^-T (D + gamma Y^T Y) R^-1, -R^-T], [-R^-1, 0]] [S^T; gamma Y^T]
// with R_ij = s_i.y_j (i <= j), D = diag(s_i.y_i), gamma = s.y / y.y of the last pair.
constexpr int kMaxLbfgsPairs = 32;
struct LbfgsState {
    int count;      // kept pairs; -1 until the first coarse CG call has built them
    int collected;  // pairs collected during that call
    int shifts;     // shifted CG calls so far (statistics)
    int negcurv;    // CG calls that ended on negative curvature (statistics)
    double gamma;
    double R[kMaxLbfgsPairs * kMaxLbfgsPairs];    // row-major, upper triangle used
    double YtY[kMaxLbfgsPairs * kMaxLbfgsPairs];  // row-major
};

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
    // CG with the L-BFGS preconditioner and the spectral shift (method 1)
    int method;            // 0: GMRES, 1: CG-QN with shift (Alg. 1)
    int m_pairs;           // secant pairs kept
    double shift_gamma;    // gamma of the shift update
    T* S_all;              // maxit * g.size: pairs collected during the first call
    T* Y_all;
    T* S;                  // m_pairs * g.size: kept pairs
    T* Y;
    LbfgsState* lb;
};

template <typename T>
jfnk_status launch_coarse(Prob prob, const CoarseArgs<T>& a, cudaStream_t st);
// count instances (2D Bratu, same coarse grid as a0), args in device memory
template <typename T>
jfnk_status launch_coarse_batched(const CoarseArgs<T>& a0, const CoarseArgs<T>* dev_args, int count, cudaStream_t st);

}  // namespace jfnk
