// Tiled element-residual kernels and their fused epilogues.
#pragma once
#include "common.cuh"

namespace jfnk {

enum class Mode : int {
    F = 0,         // out = A(w) - load ; out2 = A(w)                 (w = u)
    JV = 1,        // out = (A(u + eps v) - Au) / eps                  (Sec. 1)
    BMJ = 2,       // out = b - J v                                    (Alg. 1 restriction input)
    CHEB0 = 3,     // r = b - J s ; d = r / theta                      (Chebyshev start, s != 0)
    CHEB = 4,      // Jd ; r -= Jd ; s += d ; d' = c1 d + c2 r         (three-term step)
    CHEBLAST = 5,  // Jd ; r -= Jd ; d' = c1 d + c2 r ; s += d + d'    (last two steps fused)
};

enum class Prob : int { BRATU2 = 0, ND3 = 1, NDK3 = 2, MINSURF2 = 3, BEAM3 = 4 };

__host__ __device__ constexpr bool is_2d(Prob p) { return p == Prob::BRATU2 || p == Prob::MINSURF2; }

// Reduction epilogue: what the last block does with sum of squares of the
// reduced output (d', s or out): nothing, store the norm, or turn it into the
// FD step eps of the next action (Sec. 1 formula, mode below).
// EPS_UNIT: the next action is taken along the unit vector v/||v|| (power method):
// the step e of the slot still multiplies v while staging, and the quotient is
// divided by e ||v||, so the action returns J (v/||v||) without a normalisation pass.
enum class RedOut : int { NONE = 0, NORM = 1, EPS = 2, EPS_UNIT = 3 };

// FD step of one action, in both precisions, with its reciprocal (computed
// once by the producer of ||v|| so no kernel divides per thread).
struct EpsSlot {
    double e, inv;
    float ef, invf;
};

// Chebyshev coefficients of every step for the current lambda_l.
constexpr int kMaxChebDegree = 16;
struct ChebTable {
    double theta_inv;
    double c1[kMaxChebDegree], c2[kMaxChebDegree];
    float theta_invf;
    float c1f[kMaxChebDegree], c2f[kMaxChebDegree];
};

struct EpsParams {
    int mode;            // JFNK_EPS_PAPER / JFNK_EPS_FP32
    double n_unknowns;   // interior unknowns of the level
    const double* xstat; // device: sum|x_i| (paper) or ||x||_2 (fp32)
    int unit = 0;        // 1: slots produced from a norm are for the unit direction (EPS_UNIT)
};

template <typename T>
struct StencilArgs {
    Grid g;
    const T* u;          // base point x (Dirichlet data on the boundary)
    const T* v;          // direction (JV/BMJ/CHEB0/CHEB/CHEBLAST); null for F
    const EpsSlot* eps;  // device: FD step for v
    const T* Au;         // cached A(x)
    const T* load;       // F: subtracted (nullable)
    double load_const;   // F: constant load subtracted on interior nodes (NDK: h^3)
    const T* kappa;      // NDK: per element
    T* out;              // F, JV, BMJ: result ; CHEB0: r
    T* out2;             // F: A(w) (nullable) ; CHEB0: d
    const T* rhs;        // BMJ, CHEB0: b
    T* r;                // CHEB*: residual, updated in place
    T* s;                // CHEB*: iterate, updated in place
    T* dnew;             // CHEB, CHEBLAST: next direction (v is the current one)
    const ChebTable* cheb; // CHEB*: coefficients for the level (device)
    int cheb_step;       // CHEB*: index i of the step whose direction is v
    T node_scale;        // 3h/16 (3D) or 1 (2D)
    T lh;                // Bratu: lambda h^2 / 16; minimal surface: 1 / h^2; beam: 1 / h
    // reduction
    RedOut red;
    double* partials;
    unsigned int* counter;
    double* red_norm;    // NORM/EPS: ||.||_2 of the reduced vector (nullable)
    EpsSlot* red_eps;    // EPS: FD step of the reduced vector
    EpsParams epsp;
    int* status;         // device status word (non-finite eps)
    // scratch of the 3D kernels (nullable: then the tiled kernel runs): face
    // partial sums of the halo-free kernel, or the per-element contributions of
    // the element-parallel kernels, which run for 3D levels with n <= ep_max_n
    T* face;
    long long face_cap;
    int ep_max_n;
    int zm_min_n;        // element-parallel levels with n >= zm_min_n (> 0) march element columns along z
    int cl_min_n, cl_max_n;  // FP32 element-parallel levels with cl_min_n <= n <= cl_max_n run in one
                             // thread-block cluster (stencil_ep.cu; cl_max_n 0: never)
    int v2_threads;      // cap on the CTA size of the halo-free kernel (0: 1024; < 0: not used)
    int v3;              // FP32: the halo-free kernel's two-elements-per-thread variant (0: not used;
                         // 1 / 2: one / two CTAs per SM; other: chosen per mode)
    // adjoint kernel: per-element (dF/dkappa_e)^T v times dk_scale (nullable)
    T* dkout;
    T dk_scale;
};

// Adjoint operator: the same fused modes with J^T v (vector-Jacobian product,
// exact) in place of the FD action; Mode::JV writes J^T v.
template <typename T>
jfnk_status launch_vjp(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st);

template <typename T>
jfnk_status launch_stencil(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st);

// Chebyshev coefficients of step i for the interval [lo, hi] * lam (Saad,
// Iterative Methods for Sparse Linear Systems, Sec. 12.3):
// theta = (b+a)/2, delta = (b-a)/2, sigma = theta/delta, rho_0 = 1/sigma,
// rho_(i+1) = 1/(2 sigma - rho_i); d_(i+1) = rho_(i+1) rho_i d_i + 2 rho_(i+1)/delta r_(i+1).
__host__ __device__ inline void cheb_coeffs(double lam, double lo, double hi, int i, double& theta,
                                            double& c1, double& c2) {
    double a = lo * lam, b = hi * lam;
    theta = 0.5 * (b + a);
    double delta = 0.5 * (b - a);
    double sigma = theta / delta;
    double rho = 1.0 / sigma;
    for (int k = 0; k < i; ++k) rho = 1.0 / (2.0 * sigma - rho);
    double rho_n = 1.0 / (2.0 * sigma - rho);
    c1 = rho_n * rho;
    c2 = 2.0 * rho_n / delta;
}

__host__ __device__ inline double eps_formula(int mode, double n, double xstat, double vnorm) {
    if (!(vnorm > 0.0)) return 0.0;
    if (mode == JFNK_EPS_PAPER) {
        const double sq = 1.4901161193847656e-08;  // sqrt(2^-52)
        return sq * (n + xstat) / (n * vnorm);
    }
    const double sq32 = 3.4526698300124393e-04;    // sqrt(2^-23)
    return sq32 * (1.0 + xstat) / vnorm;
}

#ifdef __CUDACC__
// The FD-step slot of the action on a vector of norm nrm (Sec. 1 formula), with
// its reciprocal in both precisions; unit: for the direction v/||v|| (see
// RedOut::EPS_UNIT).  A non-finite step sets bit 1 of the status word and 0.
__device__ inline void set_eps_slot(EpsSlot* slot, const EpsParams& ep, double nrm, bool unit, int* status) {
    double e = eps_formula(ep.mode, ep.n_unknowns, *ep.xstat, nrm);
    double inv = e > 0.0 ? 1.0 / (unit ? e * nrm : e) : 0.0;
    if (!isfinite(e) || !isfinite(inv)) {
        if (status) atomicOr(status, 1);
        e = 0.0;
        inv = 0.0;
    }
    slot->e = e;
    slot->inv = inv;
    slot->ef = (float)e;
    slot->invf = (float)inv;
}
#endif

}  // namespace jfnk
