// jfnk_jvp_noalloc: the FD Jacobian action of jfnk_jvp for callers that cannot
// allocate device memory.
//
// jfnk_jvp keeps its reduction partials, completion counters and FD step in the
// workspace a caller allocates for a problem.  Some callers cannot do that:
// code running inside a CUDA-graph-building or plugin environment that forbids
// cudaMalloc, a host process whose device memory is fully pre-reserved by
// another allocator, or a real-time loop where an allocation would stall.  For
// them this entry point needs no problem object and no workspace: its scratch is
// the file-scope array below, which the CUDA runtime places in every device
// that loads the library and which stays allocated there until the process
// exits.
#include <cstring>

#include "common.cuh"
#include "stencil.cuh"
#include "vector.cuh"

namespace jfnk {

template <typename T>
jfnk_status launch_stencil_direct(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st);

namespace {

struct NoAllocScratch {
    RedScratch red;  // reduction partials (up to 2 * kMaxRedBlocks CTAs) and completion counters
    EpsSlot eps;     // FD step of v
    double xstat;    // sum |u_i| or ||u||_2 over interior nodes
};

constexpr size_t kNoAllocScratchBytes = (sizeof(NoAllocScratch) + 255) / 256 * 256;

// The scratch itself.  In host code this name is only a handle for
// cudaGetSymbolAddress: its device address is looked up per device below.
static __device__ __align__(256) unsigned char g_jvp_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch on the current device, looked up on every call
// (cudaGetSymbolAddress is a cheap host-side query), so that no address cached
// from an earlier context can outlive a device reset.
jfnk_status scratch_on_current_device(NoAllocScratch** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_jvp_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
        return JFNK_ERR_CUDA;
    }
    *out = reinterpret_cast<NoAllocScratch*>(p);
    return JFNK_OK;
}

template <typename T>
jfnk_status jvp_noalloc_T(int kind, int n, double lambda, const T* kappa, const T* load, const T* u, const T* Fu,
                          const T* v, T* Jv, double eps, int eps_mode, cudaStream_t st) {
    NoAllocScratch* S = nullptr;
    JFNK_TRY(scratch_on_current_device(&S));
    const int d = kind == JFNK_BRATU2D ? 2 : 3;
    const Grid g = Grid::make(d, n);
    const double h = 1.0 / n;
    // the completion counters must start at zero; an interrupted earlier call
    // could have left them otherwise
    JFNK_CUDA_TRY(cudaMemsetAsync(S->red.counter, 0, sizeof(S->red.counter), st));
    if (eps > 0.0) {
        JFNK_TRY(set_eps(&S->eps, eps, st));
    } else {
        EpsParams ep;
        ep.mode = eps_mode;
        ep.n_unknowns = (double)g.interior();
        ep.xstat = &S->xstat;
        JFNK_TRY(masked_stat<T>(g, u, eps_mode == JFNK_EPS_PAPER ? 0 : 1, &S->xstat, &S->red, st));
        JFNK_TRY(norm_to_eps<T>(g, v, ep, &S->eps, nullptr, &S->red, st));
    }
    StencilArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.node_scale = (T)(d == 3 ? 3.0 * h / 16.0 : 1.0);
    a.lh = (T)(lambda * h * h / 16.0);
    a.kappa = kappa;
    a.partials = S->red.partial;
    a.counter = &S->red.counter[1];
    a.red = RedOut::NONE;
    a.u = u;
    a.v = v;
    a.eps = &S->eps;
    a.Au = Fu;
    a.out = Jv;
    a.load = load;
    a.load_const = (kind == JFNK_NDK3D) ? h * h * h : 0.0;
    return launch_stencil_direct<T>(kind == JFNK_BRATU2D ? Prob::BRATU2 : kind == JFNK_ND3D ? Prob::ND3 : Prob::NDK3,
                                    Mode::JV, a, st);
}

}  // namespace
}  // namespace jfnk

using namespace jfnk;

jfnk_status jfnk_jvp_noalloc(int kind, int n_elem, double lambda, const void* kappa, const void* load, int dtype,
                             const void* u, const void* Fu, const void* v, void* Jv, double eps, int eps_mode,
                             void* stream) {
    if (kind < JFNK_BRATU2D || kind > JFNK_NDK3D || (dtype != JFNK_F32 && dtype != JFNK_F64) ||
        (eps_mode != JFNK_EPS_PAPER && eps_mode != JFNK_EPS_FP32) || !u || !Fu || !v || !Jv ||
        (kind == JFNK_NDK3D && !kappa)) {
        set_error("jfnk_jvp_noalloc: invalid arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    const int max_n = (kind == JFNK_BRATU2D) ? JFNK_NOALLOC_MAX_N2D : JFNK_NOALLOC_MAX_N3D;
    if (n_elem < 2 || n_elem > max_n) {
        set_error("jfnk_jvp_noalloc: n_elem %d outside [2, %d], the size its fixed scratch supports", n_elem, max_n);
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == JFNK_F64)
        return jvp_noalloc_T<double>(kind, n_elem, lambda, (const double*)kappa, (const double*)load, (const double*)u,
                                     (const double*)Fu, (const double*)v, (double*)Jv, eps, eps_mode, st);
    return jvp_noalloc_T<float>(kind, n_elem, lambda, (const float*)kappa, (const float*)load, (const float*)u,
                                (const float*)Fu, (const float*)v, (float*)Jv, eps, eps_mode, st);
}
