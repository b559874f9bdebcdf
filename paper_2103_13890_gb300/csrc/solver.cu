// Host orchestration of the Jacobian-free Newton-Krylov multigrid method and
// the C ABI of libjfnk.so (include/jfnk.h).
//
//  * Newton (Sec. 1): x^(k+1) = x^(k) + alpha dx^(k), J(x^(k)) dx = -F(x^(k)),
//    forcing ||J dx + F|| <= eta ||F|| and cubic backtracking (Sec. 3, Dennis &
//    Schnabel Sec. 6.3).
//  * Outer Krylov: right-preconditioned FGMRES(m) with classical Gram-Schmidt
//    applied twice, FD Jacobian actions in FP64 (Sec. 1).
//  * Preconditioner: the V(nu1,nu2)-cycle of Algorithm 1 with Chebyshev
//    smoothing, restriction R = I^T of b - J s, recursion, prolongation, and the
//    single-CTA GMRES coarse solve; per Newton step the iterate is projected to
//    every level with P = 2^-d I^T and lambda_l is estimated by the power method
//    (Sec. 2).  The preconditioner runs in FP32 or FP64 (opts->pc_dtype).
//
// Every step runs in the kernels of stencil.cu, vector.cu, transfer.cu and
// coarse.cu; this file only sequences launches on one stream and reads back
// the scalars that Newton and FGMRES branch on.
#include <chrono>
#include <map>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "coarse.cuh"
#include "common.cuh"
#include "stencil.cuh"
#include "transfer.cuh"
#include "vector.cuh"
#include "batch.cuh"
#include "profile.cuh"
#include "stencil_ep.cuh"
#include "beam.cuh"
#include "stencil_v2.cuh"
#include <algorithm>
#include <cstdlib>

namespace jfnk {

static thread_local std::string g_err;
static thread_local long long g_launches = 0;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
void count_launch(int k) { g_launches += k; }

namespace {
struct BoundsEntry {
    BoundsReader reader;
    const char* file;
};
std::vector<BoundsEntry>& bounds_registry() {
    static std::vector<BoundsEntry> r;
    return r;
}
}  // namespace

int register_bounds_reader(BoundsReader reader, const char* file) {
    bounds_registry().push_back({reader, file});
    return (int)bounds_registry().size();
}

struct Level {
    Grid g;
    double h;
    // preconditioner-precision vectors
    void *x, *Ax, *b, *s, *r, *d0, *d1, *t, *pv, *pw;
    // per-element coefficient of this level (NDK)
    double* kappa64;
    float* kappa32;
    // device scalars
    double* xstat_paper;  // sum |x_i| over interior
    double* xstat_fp32;   // ||x||_2 over interior
    double* lam;
    double* nrm0;
    double* nrm1;
    EpsSlot* eps_s;
    EpsSlot* eps_d;
    EpsSlot* eps_aux;
    ChebTable* cheb;
    bool pv_valid;
};

}  // namespace jfnk

struct jfnk_problem {
    jfnk_problem_desc desc;
    int d, L, n;
    std::vector<jfnk::Level> lv;
    int device;
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool bound = false;
    bool has_solver = false;
    bool adj = false;  // preconditioner and outer operator use J^T (adjoint solve)
    int pc = JFNK_F64;
    int m = 0;
    int coarse_maxit = 0;
    // finest level, FP64
    double *F64, *Au64, *load64, *Ftrial, *Autrial, *utrial, *w64, *z64, *delta, *rhs64, *tmp64;
    float* load32;
    double* V64;
    void* Z;
    double *hbuf, *ydev, *dot_partials, *nrm64, *xstat64, *scal;
    jfnk::EpsSlot* eps64;
    jfnk::RedScratch* red;
    unsigned int* counters;
    int* status;
    long long* coarse_iters;
    void* coarseV;
    double* coarseH;
    // CG-QN coarse solver: collected and kept secant pairs, compact-form state
    void *cgS_all, *cgY_all, *cgS, *cgY;
    jfnk::LbfgsState* lb;
    double* mms_tab;
    char* batch = nullptr;  // descriptor staging when this problem leads a batched solve
    size_t batch_bytes = 0;
    char* face = nullptr;  // scratch of the 3D kernels (face sums / element contributions)
    size_t face_bytes = 0;
    // 3D levels with n <= ep_max_n run the element-parallel kernels (per precision)
    int ep_max_n64 = 1 << 20;
    int ep_max_n32 = 64;
    // element-parallel levels with n >= this march element columns along z
    // (0: never), per precision.  FP64: off -- the column kernel does ~10 %
    // fewer FP64 operations but ran 5-20 % slower than one element a thread at
    // n = 64..256 (fewer warps to keep the FP64 pipe fed)
    int zm_min_n64 = 0;
    int zm_min_n32 = 0;
    // FP32 levels with cl_min_n32 <= n <= cl_max_n32 run in one thread-block
    // cluster (measured against the element-parallel pair: 22 % faster Chebyshev
    // steps at n = 16, equal at n = 32, slower than the one-CTA kernel at n = 8)
    int cl_min_n32 = 16;
    int cl_max_n32 = 16;
    // CTA-size cap of the halo-free 3D kernel (per precision)
    int v2_threads64 = 1024;
    int v2_threads32 = 1024;
    // FP32 levels on the halo-free tiling run its paired-element variant
    // (0: not used; 1 / 2: one / two CTAs per SM; 3: chosen per mode)
    int v3_f32 = 3;
    // captured V-cycle (Lf.b -> Lf.s) and the options it was captured for
    cudaGraphExec_t vgraph = nullptr;
    cudaStream_t cap_stream = nullptr;
    long long vgraph_key[16] = {0};
    long long vgraph_nF[JFNK_MAX_LEVELS] = {0};
    long long vgraph_launches = 0;
    // host counters: residual evaluations per level (FD actions included) and,
    // among them, the plain evaluations F(x) (the rest are FD actions)
    long long nF[JFNK_MAX_LEVELS];
    long long nFplain[JFNK_MAX_LEVELS];
};

namespace jfnk {

using P = jfnk_problem;

// NVTX range over a host-side phase (a level operation of the V-cycle, the
// set-up, a Krylov iteration, the line search), so that a timeline profiler
// shows the method's structure.  Without an attached profiler the calls are
// no-ops.  Ranges opened while a V-cycle is captured into a CUDA graph mark the
// capture only; graph replays carry no ranges.
struct Range {
    explicit Range(const char* fmt, int a = 0, int b = 0) {
        char buf[64];
        snprintf(buf, sizeof(buf), fmt, a, b);
        nvtxRangePushA(buf);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace planner: walks every allocation in a fixed order; with base == null
// it only sums sizes, otherwise it assigns the pointers.
struct Planner {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        size_t bytes = align256(count * sizeof(T));
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

static size_t plan(P& p, char* base, const jfnk_options* o) {
    Planner pl{base};
    const size_t esz_pc = (o && o->pc_dtype == JFNK_F32) ? 4 : 8;
    p.red = pl.take<RedScratch>(1);
    p.status = pl.take<int>(64);
    p.counters = pl.take<unsigned int>(64);
    p.scal = pl.take<double>(64);
    p.eps64 = pl.take<EpsSlot>(4);
    p.nrm64 = pl.take<double>(8);
    p.xstat64 = pl.take<double>(8);
    p.coarse_iters = pl.take<long long>(8);
    for (int l = 0; l <= p.L; ++l) {
        Level& L = p.lv[l];
        L.xstat_paper = pl.take<double>(1);
        L.xstat_fp32 = pl.take<double>(1);
        L.lam = pl.take<double>(1);
        L.nrm0 = pl.take<double>(1);
        L.nrm1 = pl.take<double>(1);
        L.eps_s = pl.take<EpsSlot>(1);
        L.eps_d = pl.take<EpsSlot>(1);
        L.eps_aux = pl.take<EpsSlot>(1);
        L.cheb = pl.take<ChebTable>(1);
        if (p.desc.kind == JFNK_NDK3D) {
            const size_t ne = (size_t)L.g.n * L.g.n * L.g.n;
            L.kappa64 = pl.take<double>(ne);
            L.kappa32 = pl.take<float>(ne);
        } else {
            L.kappa64 = nullptr;
            L.kappa32 = nullptr;
        }
    }
    const Grid& gf = p.lv[p.L].g;
    const size_t N = (size_t)gf.size;
    if (const char* e = getenv("JFNK_EP3D_MAX_N_F64")) p.ep_max_n64 = atoi(e);
    if (const char* e = getenv("JFNK_EP3D_MAX_N_F32")) p.ep_max_n32 = atoi(e);
    if (const char* e = getenv("JFNK_ZM3D_MIN_N_F64")) p.zm_min_n64 = atoi(e);
    if (const char* e = getenv("JFNK_ZM3D_MIN_N_F32")) p.zm_min_n32 = atoi(e);
    if (const char* e = getenv("JFNK_EP3D_CLUSTER_MIN_N")) p.cl_min_n32 = atoi(e);
    if (const char* e = getenv("JFNK_EP3D_CLUSTER_MAX_N")) p.cl_max_n32 = atoi(e);
    // the cluster kernels' attributes are set here, outside any graph capture
    if (p.cl_max_n32 > 0 && !ep3d_cluster_init()) p.cl_max_n32 = 0;
    if (const char* e = getenv("JFNK_V2_THREADS_F64")) p.v2_threads64 = atoi(e);
    if (const char* e = getenv("JFNK_V2_THREADS_F32")) p.v2_threads32 = atoi(e);
    if (const char* e = getenv("JFNK_V3_F32")) p.v3_f32 = atoi(e);
    long long face = 0;
    for (int l = 0; l <= p.L; ++l) {
        const Grid& g = p.lv[l].g;
        face = std::max(face, v2_face_count(g, p.v2_threads64));
        face = std::max(face, v2_face_count(g, p.v2_threads32));
        if (p.v3_f32) {
            face = std::max(face, v3_face_count(g, p.v2_threads32, 1));
            face = std::max(face, v3_face_count(g, p.v2_threads32, 2));
        }
        face = std::max(face, beam_scratch_count(g));
        // (in doubles; an FP32 level's T entries take half as many bytes)
        if (g.n <= std::max(p.ep_max_n64, p.ep_max_n32)) face = std::max(face, ep3d_scratch_count(g));
        if (p.zm_min_n64 > 0 && g.n >= p.zm_min_n64) face = std::max(face, ep3d_scratch_need(g, true));
        if (p.zm_min_n32 > 0 && g.n >= p.zm_min_n32) face = std::max(face, (ep3d_scratch_need(g, true) + 1) / 2);
    }
    p.face_bytes = (size_t)face * sizeof(double);
    p.face = face > 0 ? pl.take<char>(p.face_bytes) : nullptr;
    p.F64 = pl.take<double>(N);
    p.Au64 = pl.take<double>(N);
    p.tmp64 = pl.take<double>(N);
    if (p.desc.kind == JFNK_ND3D) {
        p.load64 = pl.take<double>(N);
        p.load32 = pl.take<float>(N);
        p.mms_tab = pl.take<double>(3 * (size_t)gf.nx);
    } else {
        p.load64 = nullptr;
        p.load32 = nullptr;
        p.mms_tab = nullptr;
    }
    if (o) {
        for (int l = 0; l <= p.L; ++l) {
            Level& L = p.lv[l];
            const size_t n = (size_t)L.g.size;
            void** vecs[] = {&L.x, &L.Ax, &L.b, &L.s, &L.r, &L.d0, &L.d1, &L.t, &L.pv, &L.pw};
            for (void** v : vecs) *v = pl.take<char>(n * esz_pc);
        }
        const int m = o->restart;
        p.V64 = pl.take<double>((size_t)(m + 1) * N);
        p.Z = pl.take<char>((size_t)m * N * esz_pc);
        p.Ftrial = pl.take<double>(N);
        p.Autrial = pl.take<double>(N);
        p.utrial = pl.take<double>(N);
        p.w64 = pl.take<double>(N);
        p.z64 = pl.take<double>(N);
        p.delta = pl.take<double>(N);
        p.rhs64 = pl.take<double>(N);
        p.hbuf = pl.take<double>(4 * (size_t)(m + 2));
        p.ydev = pl.take<double>((size_t)(m + 2));
        p.dot_partials = pl.take<double>((size_t)(m + 9) * kDotBlocks);
        const Grid& g0 = p.lv[0].g;
        const int cm = o->coarse_maxit > 0 ? o->coarse_maxit : (int)g0.interior();
        p.coarseV = pl.take<char>((size_t)(cm + 1) * g0.size * esz_pc);
        p.coarseH = pl.take<double>((size_t)(cm + 1) * cm);
        p.cgS_all = pl.take<char>((size_t)cm * g0.size * esz_pc);
        p.cgY_all = pl.take<char>((size_t)cm * g0.size * esz_pc);
        p.cgS = pl.take<char>((size_t)kMaxLbfgsPairs * g0.size * esz_pc);
        p.cgY = pl.take<char>((size_t)kMaxLbfgsPairs * g0.size * esz_pc);
        p.lb = pl.take<LbfgsState>(1);
        // descriptor staging of batched solves led by this problem
        p.batch_bytes = (size_t)32 << 20;
        p.batch = pl.take<char>(p.batch_bytes);
    }
    return pl.off;
}

// ---------------------------------------------------------------------------
static EpsParams eps_params(P& p, int l, int mode) {
    Level& L = p.lv[l];
    EpsParams e;
    e.mode = mode;
    e.n_unknowns = (double)L.g.interior();
    e.xstat = (mode == JFNK_EPS_PAPER) ? L.xstat_paper : L.xstat_fp32;
    return e;
}

static Prob prob_of(const P& p) {
    switch (p.desc.kind) {
        case JFNK_BRATU2D: return Prob::BRATU2;
        case JFNK_MINSURF2D: return Prob::MINSURF2;
        case JFNK_BEAM3D: return Prob::BEAM3;
        case JFNK_ND3D: return Prob::ND3;
        default: return Prob::NDK3;
    }
}

// element parameter: Bratu lambda h^2 / 16, minimal surface 1 / h^2, beam 1 / h
static double lh_of(const P& p, double h) {
    if (p.desc.kind == JFNK_BEAM3D) return 1.0 / h;
    return p.desc.kind == JFNK_MINSURF2D ? 1.0 / (h * h) : p.desc.lambda * h * h / 16.0;
}

// factor applied to the summed element contributions of a node: 3h/16 for the
// scaled 3D scalar elements, 1 where the element returns the integral itself
static double node_scale_of(const P& p, double h) {
    return (p.d == 3 && p.desc.kind != JFNK_BEAM3D) ? 3.0 * h / 16.0 : 1.0;
}

template <typename T>
static const T* kappa_of(P& p, int l);
template <>
const double* kappa_of<double>(P& p, int l) { return p.lv[l].kappa64; }
template <>
const float* kappa_of<float>(P& p, int l) { return p.lv[l].kappa32; }

template <typename T>
static const T* load_of(P& p);
template <>
const double* load_of<double>(P& p) { return p.load64; }
template <>
const float* load_of<float>(P& p) { return p.load32; }

template <typename T>
static StencilArgs<T> base_args(P& p, int l) {
    Level& L = p.lv[l];
    StencilArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = L.g;
    a.node_scale = (T)node_scale_of(p, L.h);
    a.lh = (T)lh_of(p, L.h);
    a.kappa = kappa_of<T>(p, l);
    a.partials = p.red->partial;
    a.counter = &p.red->counter[1];
    a.status = p.status;
    a.red = RedOut::NONE;
    a.face = reinterpret_cast<T*>(p.face);
    a.face_cap = (long long)(p.face_bytes / sizeof(T));
    a.ep_max_n = sizeof(T) == 8 ? p.ep_max_n64 : p.ep_max_n32;
    a.zm_min_n = sizeof(T) == 8 ? p.zm_min_n64 : p.zm_min_n32;
    a.cl_min_n = sizeof(T) == 4 ? p.cl_min_n32 : 0;
    a.cl_max_n = sizeof(T) == 4 ? p.cl_max_n32 : 0;
    a.v2_threads = sizeof(T) == 8 ? p.v2_threads64 : p.v2_threads32;
    a.v3 = sizeof(T) == 4 ? p.v3_f32 : 0;
    return a;
}

// Operator of the multigrid cycle: the FD action of F (forward) or the exact
// vector-Jacobian product J^T v (adjoint solve).
template <typename T>
static jfnk_status launch_op(P& p, Mode m, const StencilArgs<T>& a, cudaStream_t st) {
    if (p.adj) return launch_vjp<T>(prob_of(p), m, a, st);
    return launch_stencil<T>(prob_of(p), m, a, st);
}

template <typename T>
static T* as(void* v) {
    return reinterpret_cast<T*>(v);
}

// ---------------------------------------------------------------------------
// Preconditioner (precision T)
// ---------------------------------------------------------------------------
template <typename T>
static jfnk_status smooth(P& p, const jfnk_options& o, int l, const T* b, T* s, int nu, bool s_zero,
                          cudaStream_t st) {
    Level& L = p.lv[l];
    const int k = o.cheb_degree;
    const EpsParams ep = eps_params(p, l, o.eps_mode_pc);
    Range rg("smooth l%d nu%d", l, nu);
    for (int app = 0; app < nu; ++app) {
        T* dc = as<T>(L.d0);
        T* dn = as<T>(L.d1);
        if (app == 0 && s_zero) {
            JFNK_TRY(cheb_start_zero<T>(L.g, b, as<T>(L.r), dc, L.cheb, ep, L.eps_d, p.red, st));
        } else {
            StencilArgs<T> a = base_args<T>(p, l);
            a.u = as<T>(L.x);
            a.v = s;
            a.eps = L.eps_s;
            a.Au = as<T>(L.Ax);
            a.rhs = b;
            a.out = as<T>(L.r);
            a.out2 = dc;
            a.cheb = L.cheb;
            a.cheb_step = 0;
            a.red = RedOut::EPS;
            a.red_eps = L.eps_d;
            a.epsp = ep;
            JFNK_TRY(launch_op<T>(p, Mode::CHEB0, a, st));
            p.nF[l]++;
        }
        if (k == 1) {
            JFNK_TRY(add_inplace<T>(s, dc, L.g.size, st));
            JFNK_TRY(norm_to_eps<T>(L.g, s, ep, L.eps_s, nullptr, p.red, st));
            continue;
        }
        for (int i = 0; i <= k - 2; ++i) {
            StencilArgs<T> a = base_args<T>(p, l);
            a.u = as<T>(L.x);
            a.v = dc;
            a.eps = L.eps_d;
            a.Au = as<T>(L.Ax);
            a.r = as<T>(L.r);
            a.s = s;
            a.dnew = dn;
            a.cheb = L.cheb;
            a.cheb_step = i;
            a.red = RedOut::EPS;
            a.epsp = ep;
            if (i < k - 2) {
                a.red_eps = L.eps_d;
                JFNK_TRY(launch_op<T>(p, Mode::CHEB, a, st));
            } else {
                a.red_eps = L.eps_s;
                JFNK_TRY(launch_op<T>(p, Mode::CHEBLAST, a, st));
            }
            p.nF[l]++;
            T* tmp = dc;
            dc = dn;
            dn = tmp;
        }
    }
    return JFNK_OK;
}

template <typename T>
static jfnk_status coarse_solve(P& p, const jfnk_options& o, const T* b, T* s, cudaStream_t st) {
    Range rg("coarse solve");
    Level& L = p.lv[0];
    CoarseArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = L.g;
    a.x = as<T>(L.x);
    a.Ax = as<T>(L.Ax);
    a.b = b;
    a.s = s;
    a.kappa = kappa_of<T>(p, 0);
    a.lh = (T)lh_of(p, L.h);
    a.node_scale = (T)node_scale_of(p, L.h);
    a.eps_mode = o.eps_mode_pc;
    a.n_unknowns = (double)L.g.interior();
    a.xstat = (o.eps_mode_pc == JFNK_EPS_PAPER) ? L.xstat_paper : L.xstat_fp32;
    a.tol = o.coarse_tol;
    a.tol_abs = o.coarse_tol_mode;
    a.maxit = p.coarse_maxit;
    a.V = as<T>(p.coarseV);
    a.H = p.coarseH;
    a.iters = p.coarse_iters;
    a.adjoint = p.adj ? 1 : 0;
    // the adjoint solve keeps GMRES (its operator J^T is not the Hessian of an energy)
    a.method = (o.coarse_method == JFNK_COARSE_CGQN && !p.adj) ? 1 : 0;
    a.m_pairs = o.lbfgs_pairs;
    a.shift_gamma = o.shift_gamma;
    a.S_all = as<T>(p.cgS_all);
    a.Y_all = as<T>(p.cgY_all);
    a.S = as<T>(p.cgS);
    a.Y = as<T>(p.cgY);
    a.lb = p.lb;
    return launch_coarse<T>(prob_of(p), a, st);
}

template <typename T>
static jfnk_status vcycle(P& p, const jfnk_options& o, int l, T* b, T* s, cudaStream_t st) {
    if (l == 0) return coarse_solve<T>(p, o, b, s, st);
    Level& L = p.lv[l];
    Level& C = p.lv[l - 1];
    JFNK_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(T) * L.g.size, st));
    JFNK_TRY(smooth<T>(p, o, l, b, s, o.nu_pre, true, st));
    // r_(l-1) = R (b - J s)        (Alg. 1, restriction of the residual)
    if (o.nu_pre == 0) JFNK_TRY(set_eps(L.eps_s, 0.0, st));
    {
        Range rg("restrict l%d", l);
        StencilArgs<T> a = base_args<T>(p, l);
        a.u = as<T>(L.x);
        a.v = s;
        a.eps = L.eps_s;
        a.Au = as<T>(L.Ax);
        a.rhs = b;
        a.out = as<T>(L.t);
        JFNK_TRY(launch_op<T>(p, Mode::BMJ, a, st));
        p.nF[l]++;
        JFNK_TRY(restrict_to<T>(L.g, C.g, as<T>(L.t), as<T>(C.b), false, st));
    }
    // c_(l-1) = MG(x_(l-1), F(x_(l-1)), r_(l-1), l-1)
    JFNK_TRY(vcycle<T>(p, o, l - 1, as<T>(C.b), as<T>(C.s), st));
    // s += I c
    {
        Range rg("prolong l%d", l);
        JFNK_TRY(prolong_add<T>(C.g, L.g, as<T>(C.s), s, st));
        JFNK_TRY(norm_to_eps<T>(L.g, s, eps_params(p, l, o.eps_mode_pc), L.eps_s, nullptr, p.red, st));
    }
    JFNK_TRY(smooth<T>(p, o, l, b, s, o.nu_post, false, st));
    return JFNK_OK;
}

// One V-cycle Lf.b -> Lf.s replayed from a CUDA graph.  Every launch of the
// cycle reads its scalars (FD steps, Chebyshev coefficients, lambda_l) from
// device memory, so the captured sequence stays valid across Newton steps; it
// is recaptured when the options that shape it change.
template <typename T>
static jfnk_status vcycle_graph(P& p, const jfnk_options& o, cudaStream_t st) {
    long long key[16] = {o.nu_pre, o.nu_post, o.cheb_degree, o.pc_dtype, o.eps_mode_pc, p.coarse_maxit, 0,
                         o.coarse_tol_mode, p.adj ? 1 : 0, (long long)sizeof(T), 1, o.coarse_method,
                         o.lbfgs_pairs, 0, 0, 0};
    memcpy(&key[6], &o.coarse_tol, sizeof(double));
    memcpy(&key[13], &o.shift_gamma, sizeof(double));
    if (p.vgraph && memcmp(key, p.vgraph_key, sizeof(key)) != 0) {
        cudaGraphExecDestroy(p.vgraph);
        p.vgraph = nullptr;
    }
    Level& Lf = p.lv[p.L];
    if (!p.vgraph) {
        if (!p.cap_stream) JFNK_CUDA_TRY(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
        long long nF0[JFNK_MAX_LEVELS];
        memcpy(nF0, p.nF, sizeof(nF0));
        const long long l0 = g_launches;
        JFNK_CUDA_TRY(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
        jfnk_status s = vcycle<T>(p, o, p.L, as<T>(Lf.b), as<T>(Lf.s), p.cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
        if (s != JFNK_OK) {
            if (e == cudaSuccess && graph) cudaGraphDestroy(graph);
            return s;
        }
        JFNK_CUDA_TRY(e);
        cudaError_t ei = cudaGraphInstantiate(&p.vgraph, graph, 0);
        cudaGraphDestroy(graph);
        JFNK_CUDA_TRY(ei);
        for (int l = 0; l < JFNK_MAX_LEVELS; ++l) p.vgraph_nF[l] = p.nF[l] - nF0[l];
        memcpy(p.nF, nF0, sizeof(nF0));  // the captured launches have not run
        p.vgraph_launches = g_launches - l0;
        g_launches = l0;
        memcpy(p.vgraph_key, key, sizeof(key));
    }
    JFNK_CUDA_TRY(cudaGraphLaunch(p.vgraph, st));
    for (int l = 0; l < JFNK_MAX_LEVELS; ++l) p.nF[l] += p.vgraph_nF[l];
    g_launches += p.vgraph_launches;
    return JFNK_OK;
}

// x_L = u, x_(l-1) = P x_l, A(x_l), statistics for eps, power method (Sec. 2)
template <typename T>
// au_fine (nullable): A(u) at the finest level, already evaluated in FP64 for
// this u (the Newton residual); an FP64 hierarchy copies it instead of
// evaluating the same kernel on the same input again.
static jfnk_status mg_setup_T(P& p, const jfnk_options& o, const double* u, int newton_step, cudaStream_t st,
                              const double* au_fine = nullptr) {
    Range rg("mg setup (Newton step %d)", newton_step);
    Level& Lf = p.lv[p.L];
    if (newton_step == 0 && p.lb) {
        // the L-BFGS preconditioner of the coarse CG is built during the first
        // coarse solve of a Newton run (Sec. 3) and kept until the next run
        LbfgsState h;
        memset(&h, 0, sizeof(h));
        h.count = -1;
        JFNK_CUDA_TRY(cudaMemcpyAsync(p.lb, &h, 4 * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    JFNK_TRY((cast_copy<T, double>(as<T>(Lf.x), u, Lf.g.size, st)));
    for (int l = p.L; l >= 1; --l)
        JFNK_TRY(restrict_to<T>(p.lv[l].g, p.lv[l - 1].g, as<T>(p.lv[l].x), as<T>(p.lv[l - 1].x), true, st));
    for (int l = 0; l <= p.L; ++l) {
        Level& L = p.lv[l];
        if (l == p.L && au_fine && sizeof(T) == 8) {
            JFNK_CUDA_TRY(cudaMemcpyAsync(L.Ax, au_fine, sizeof(double) * L.g.size, cudaMemcpyDeviceToDevice, st));
        } else {
            StencilArgs<T> a = base_args<T>(p, l);
            a.u = as<T>(L.x);
            a.out = as<T>(L.Ax);
            JFNK_TRY(launch_stencil<T>(prob_of(p), Mode::F, a, st));
            p.nF[l]++;
            p.nFplain[l]++;
        }
        JFNK_TRY(masked_stat<T>(L.g, as<T>(L.x), 0, L.xstat_paper, p.red, st));
        JFNK_TRY(masked_stat<T>(L.g, as<T>(L.x), 1, L.xstat_fp32, p.red, st));
    }
    // Power method on every smoothed level.  The levels are independent, so
    // iteration i is issued for every level still running before the host
    // reads their estimates: with the stopping rule on, one synchronisation
    // per iteration instead of one per level and iteration.  Each level runs
    // the same kernels in the same order as it would alone.
    std::vector<int> active;
    for (int l = 1; l <= p.L; ++l) {
        Level& L = p.lv[l];
        const EpsParams ep = eps_params(p, l, o.eps_mode_pc);
        if (newton_step == 0 || !L.pv_valid) JFNK_TRY(splitmix_start<T>(L.g, as<T>(L.pv), o.seed, l, st));
        if (!p.adj) {
            // FD power iteration along unit vectors without normalisation passes:
            // each action takes v/||v|| (RedOut::EPS_UNIT), so lambda = ||J v/||v|| ||
            // is the action's own output norm and the output is the next v
            EpsParams epu = ep;
            epu.unit = 1;
            JFNK_TRY(norm_to_eps<T>(L.g, as<T>(L.pv), epu, L.eps_aux, L.nrm0, p.red, st));
        } else {
            // adjoint operator (exact J^T v): normalise explicitly
            JFNK_TRY(norm_to_eps<T>(L.g, as<T>(L.pv), ep, L.eps_aux, L.nrm0, p.red, st));
            JFNK_TRY(scale_inplace_inv<T>(as<T>(L.pv), L.g.size, L.nrm0, st));
        }
        active.push_back(l);
    }
    auto iterate = [&](int l) -> jfnk_status {
        Level& L = p.lv[l];
        StencilArgs<T> a = base_args<T>(p, l);
        a.u = as<T>(L.x);
        a.v = as<T>(L.pv);
        a.eps = L.eps_aux;
        a.Au = as<T>(L.Ax);
        a.out = as<T>(L.pw);
        if (!p.adj) {
            EpsParams epu = eps_params(p, l, o.eps_mode_pc);
            epu.unit = 1;
            a.red = RedOut::EPS_UNIT;
            a.red_norm = L.lam;
            a.red_eps = L.eps_aux;
            a.epsp = epu;
            JFNK_TRY(launch_stencil<T>(prob_of(p), Mode::JV, a, st));
        } else {
            JFNK_TRY(norm_to_eps<T>(L.g, as<T>(L.pv), eps_params(p, l, o.eps_mode_pc), L.eps_aux, L.nrm0, p.red,
                                    st));
            a.red = RedOut::NORM;
            a.red_norm = L.nrm1;
            JFNK_TRY(launch_op<T>(p, Mode::JV, a, st));
            // lambda = ||J v|| / ||v||; v <- J v / ||J v||
            JFNK_TRY(ratio_scalar(L.lam, L.nrm1, L.nrm0, st));
            JFNK_TRY(scale_inplace_inv<T>(as<T>(L.pw), L.g.size, L.nrm1, st));
        }
        p.nF[l]++;
        std::swap(L.pv, L.pw);
        return JFNK_OK;
    };
    std::vector<double> lam_prev(p.L + 1, 0.0), lam_now(p.L + 1, 0.0);
    for (int it = 0; it < o.power_iters && !active.empty(); ++it) {
        for (int l : active) JFNK_TRY(iterate(l));
        if (o.power_tol > 0.0) {
            for (int l : active)
                JFNK_CUDA_TRY(cudaMemcpyAsync(&lam_now[l], p.lv[l].lam, sizeof(double), cudaMemcpyDeviceToHost, st));
            JFNK_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<int> still;
            for (int l : active) {
                const bool done = it > 0 && std::fabs(lam_now[l] - lam_prev[l]) < o.power_tol * lam_now[l];
                lam_prev[l] = lam_now[l];
                if (!done) still.push_back(l);
            }
            active.swap(still);
        }
    }
    for (int l = 1; l <= p.L; ++l) {
        Level& L = p.lv[l];
        L.pv_valid = true;
        JFNK_TRY(cheb_table(L.lam, o.cheb_lo, o.cheb_hi, o.cheb_degree, L.cheb, p.status, st));
    }
    return JFNK_OK;
}

// F = A(u) - load (finest, FP64) and A(u)
static jfnk_status residual64(P& p, const double* u, double* F, double* Au, cudaStream_t st) {
    StencilArgs<double> a = base_args<double>(p, p.L);
    a.u = u;
    a.out = F;
    a.out2 = Au;
    a.load = p.load64;
    a.load_const = (p.desc.kind == JFNK_NDK3D) ? std::pow(p.lv[p.L].h, 3) : 0.0;
    p.nF[p.L]++;
    p.nFplain[p.L]++;
    return launch_stencil<double>(prob_of(p), Mode::F, a, st);
}

static jfnk_status read_norm(P& p, const double* v, double* host, cudaStream_t st) {
    JFNK_TRY(masked_stat<double>(p.lv[p.L].g, v, 1, p.nrm64, p.red, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(host, p.nrm64, sizeof(double), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    return JFNK_OK;
}

// w = J(u) v in FP64 with the paper's eps (Sec. 1); Au = A(u).  In the adjoint
// solve w = J(u)^T v (exact vector-Jacobian product).
static jfnk_status jv64(P& p, const double* u, const double* Au, const double* v, double* w, cudaStream_t st) {
    const Grid& g = p.lv[p.L].g;
    if (p.adj) {
        StencilArgs<double> a = base_args<double>(p, p.L);
        a.u = u;
        a.v = v;
        a.out = w;
        p.nF[p.L]++;
        return launch_vjp<double>(prob_of(p), Mode::JV, a, st);
    }
    EpsParams ep;
    ep.mode = JFNK_EPS_PAPER;
    ep.n_unknowns = (double)g.interior();
    ep.xstat = p.xstat64;
    JFNK_TRY(norm_to_eps<double>(g, v, ep, p.eps64, nullptr, p.red, st));
    StencilArgs<double> a = base_args<double>(p, p.L);
    a.u = u;
    a.v = v;
    a.eps = p.eps64;
    a.Au = Au;
    a.out = w;
    p.nF[p.L]++;
    return launch_stencil<double>(prob_of(p), Mode::JV, a, st);
}

static void givens(double a, double b, double& c, double& s) {
    if (b == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    const double r = std::hypot(a, b);
    c = a / r;
    s = b / r;
}

// What FGMRES leaves for the line-search slope: the Arnoldi cycles run and,
// from the last cycle, beta = ||r|| at its start and (Hbar y)_0, the first entry
// of the unrotated Hessenberg matrix times the least-squares solution.  After a
// single cycle from delta = 0 (v_0 = rhs / beta) the Arnoldi relation
// J Z y = V Hbar y gives rhs . (J delta) = beta (Hbar y)_0 from the FD actions
// already applied.
struct ArnoldiSlope {
    int cycles = 0;
    double beta = 0.0, Hy0 = 0.0;
};

// FGMRES(m): J(u) delta = rhs64 to ||rhs - J delta|| <= eta ||rhs||, right-
// preconditioned by one V-cycle per iteration.
template <typename T>
static jfnk_status fgmres(P& p, const jfnk_options& o, const double* u, double eta, int& its, cudaStream_t st,
                          ArnoldiSlope* slope = nullptr) {
    const Grid& g = p.lv[p.L].g;
    const long long N = g.size;
    const int m = o.restart;
    Level& Lf = p.lv[p.L];
    its = 0;
    JFNK_CUDA_TRY(cudaMemsetAsync(p.delta, 0, sizeof(double) * N, st));
    double beta0 = 0.0;
    JFNK_TRY(read_norm(p, p.rhs64, &beta0, st));
    if (!(beta0 > 0.0)) return JFNK_OK;
    if (!std::isfinite(beta0)) {
        set_error("non-finite right-hand side in FGMRES");
        return JFNK_ERR_NONFINITE;
    }
    const double target = eta * beta0;
    JFNK_CUDA_TRY(cudaMemcpyAsync(p.tmp64, p.rhs64, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    double beta = beta0;
    std::vector<double> H((size_t)(m + 1) * m), Hraw((size_t)(m + 1) * m), gv(m + 1), cs(m), sn(m), y(m),
        hh(2 * (m + 2));
    T* Z = as<T>(p.Z);
    int cycles = 0;
    while (true) {
        cycles++;
        // V_0 = r / beta
        JFNK_CUDA_TRY(cudaMemcpyAsync(p.scal, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
        JFNK_TRY(scale_by_inv(p.V64, p.tmp64, N, p.scal, st));
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int k = 0;
        double res = beta;
        bool stop = false;
        for (int j = 0; j < m; ++j) {
            Range rg("FGMRES iteration %d", its);
            double* vj = p.V64 + (size_t)j * N;
            T* zj = Z + (size_t)j * N;
            // z_j = MG(v_j)
            JFNK_TRY((cast_copy<T, double>(as<T>(Lf.b), vj, N, st)));
            if (o.use_graph && !prof_on()) {
                JFNK_TRY(vcycle_graph<T>(p, o, st));
                JFNK_CUDA_TRY(cudaMemcpyAsync(zj, Lf.s, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
            } else {
                JFNK_TRY(vcycle<T>(p, o, p.L, as<T>(Lf.b), zj, st));
            }
            // w = J z_j  (FP64)
            const double* z64 = nullptr;
            if (sizeof(T) == 8) {
                z64 = reinterpret_cast<const double*>(zj);
            } else {
                JFNK_TRY((cast_copy<double, T>(p.z64, zj, N, st)));
                z64 = p.z64;
            }
            JFNK_TRY(jv64(p, u, p.Au64, z64, p.w64, st));
            // CGS2
            JFNK_TRY(multi_dot(p.w64, p.V64, N, N, j + 1, p.hbuf, p.dot_partials, &p.counters[2], st));
            JFNK_TRY(multi_axpy_sub(p.w64, p.V64, N, N, j + 1, p.hbuf, st));
            JFNK_TRY(multi_dot(p.w64, p.V64, N, N, j + 1, p.hbuf + (m + 2), p.dot_partials, &p.counters[2], st));
            JFNK_TRY(multi_axpy_sub(p.w64, p.V64, N, N, j + 1, p.hbuf + (m + 2), st));
            JFNK_TRY(masked_stat<double>(g, p.w64, 1, p.hbuf + 2 * (m + 2), p.red, st));
            JFNK_CUDA_TRY(cudaMemcpyAsync(hh.data(), p.hbuf, sizeof(double) * 2 * (m + 2), cudaMemcpyDeviceToHost, st));
            double hn = 0.0;
            JFNK_CUDA_TRY(cudaMemcpyAsync(&hn, p.hbuf + 2 * (m + 2), sizeof(double), cudaMemcpyDeviceToHost, st));
            JFNK_CUDA_TRY(cudaStreamSynchronize(st));
            double* col = &H[(size_t)j * (m + 1)];
            for (int i = 0; i <= j; ++i) col[i] = hh[i] + hh[(m + 2) + i];
            col[j + 1] = hn;
            for (int i = 0; i <= j + 1; ++i) Hraw[(size_t)j * (m + 1) + i] = col[i];
            if (!std::isfinite(hn)) {
                set_error("non-finite Arnoldi entry in FGMRES");
                return JFNK_ERR_NONFINITE;
            }
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            givens(col[j], col[j + 1], cs[j], sn[j]);
            col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
            col[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            res = std::fabs(gv[j + 1]);
            k = j + 1;
            its++;
            if (res <= target || its >= o.max_linear || hn == 0.0) {
                stop = true;
                break;
            }
            JFNK_TRY(scale_by_inv(p.V64 + (size_t)(j + 1) * N, p.w64, N, p.hbuf + 2 * (m + 2), st));
        }
        // y = H^-1 g, delta += Z y.  A zero diagonal entry of the rotated
        // Hessenberg matrix means the Krylov space stopped growing with the
        // preconditioned direction mapped to zero (J z_j = 0 in its span): the
        // least-squares problem is singular and there is no update to take.
        for (int i = k - 1; i >= 0; --i) {
            const double hii = H[(size_t)i * (m + 1) + i];
            if (hii == 0.0) {
                set_error("FGMRES breakdown: singular Hessenberg matrix at column %d (residual %.3e)", i, res);
                return JFNK_ERR_BREAKDOWN;
            }
            double t = gv[i];
            for (int q = i + 1; q < k; ++q) t -= H[(size_t)q * (m + 1) + i] * y[q];
            y[i] = t / hii;
        }
        JFNK_CUDA_TRY(cudaMemcpyAsync(p.ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        JFNK_TRY(combine<T>(p.delta, Z, N, N, k, p.ydev, st));
        if (slope) {
            double hy0 = 0.0;
            for (int q = 0; q < k; ++q) hy0 += Hraw[(size_t)q * (m + 1)] * y[q];
            slope->cycles = cycles;
            slope->beta = beta;
            slope->Hy0 = hy0;
        }
        if (stop) break;
        // restart: r = rhs - J delta
        JFNK_TRY(jv64(p, u, p.Au64, p.delta, p.w64, st));
        JFNK_TRY(add_scaled(p.tmp64, p.rhs64, -1.0, p.w64, N, st));
        JFNK_TRY(read_norm(p, p.tmp64, &beta, st));
        if (beta <= target) break;
    }
    return JFNK_OK;
}

// z = MG(r) for the outer Krylov method: r (FP64) -> preconditioner precision
// -> V-cycle (graph replay when enabled) -> z (FP64)
template <typename T>
static jfnk_status apply_mg64(P& p, const jfnk_options& o, const double* r, double* z, cudaStream_t st) {
    Level& Lf = p.lv[p.L];
    const long long N = Lf.g.size;
    JFNK_TRY((cast_copy<T, double>(as<T>(Lf.b), r, N, st)));
    if (o.use_graph && !prof_on()) {
        JFNK_TRY(vcycle_graph<T>(p, o, st));
    } else {
        JFNK_TRY(vcycle<T>(p, o, p.L, as<T>(Lf.b), as<T>(Lf.s), st));
    }
    return cast_copy<double, T>(z, as<T>(Lf.s), N, st);
}

static jfnk_status dot2(P& p, const double* a, const double* b, const double* c, const double* d, double* out,
                        cudaStream_t st) {
    const long long N = p.lv[p.L].g.size;
    JFNK_TRY(multi_dot(a, b, N, N, 1, p.hbuf, p.dot_partials, &p.counters[2], st));
    if (c) JFNK_TRY(multi_dot(c, d, N, N, 1, p.hbuf + 1, p.dot_partials, &p.counters[2], st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(out, p.hbuf, sizeof(double) * (c ? 2 : 1), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    return JFNK_OK;
}

// The paper's outer Krylov method (Sec. 3): preconditioned CG for J delta = -F
// from delta = 0 with z = MG(r), stopped at ||r|| <= eta ||F|| or max_linear
// iterations.  On negative curvature p.Jp <= 0 it returns the current iterate,
// or the first search direction at the first iteration (Nocedal & Wright,
// Numerical Optimization, Alg. 7.1).  Vectors: delta, r = tmp64, z = z64,
// p = V64 (the FGMRES basis is unused), q = J p = w64.
template <typename T>
static jfnk_status pcg(P& p, const jfnk_options& o, const double* u, double eta, int& its, int& negc,
                       cudaStream_t st) {
    const long long N = p.lv[p.L].g.size;
    double* pd = p.V64;
    its = 0;
    negc = 0;
    JFNK_CUDA_TRY(cudaMemsetAsync(p.delta, 0, sizeof(double) * N, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(p.tmp64, p.rhs64, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    double res = 0.0;
    JFNK_TRY(read_norm(p, p.tmp64, &res, st));
    if (!(res > 0.0)) return JFNK_OK;
    if (!std::isfinite(res)) {
        set_error("non-finite right-hand side in CG");
        return JFNK_ERR_NONFINITE;
    }
    const double target = eta * res;
    JFNK_TRY(apply_mg64<T>(p, o, p.tmp64, p.z64, st));
    double rz = 0.0;
    JFNK_TRY(dot2(p, p.tmp64, p.z64, nullptr, nullptr, &rz, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(pd, p.z64, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    for (int it = 1; it <= o.max_linear; ++it) {
        JFNK_TRY(jv64(p, u, p.Au64, pd, p.w64, st));
        double pq = 0.0;
        JFNK_TRY(dot2(p, pd, p.w64, nullptr, nullptr, &pq, st));
        its = it;
        if (!std::isfinite(pq)) {
            set_error("non-finite curvature in CG");
            return JFNK_ERR_NONFINITE;
        }
        if (pq <= 0.0) {
            negc = 1;
            if (it == 1) JFNK_CUDA_TRY(cudaMemcpyAsync(p.delta, pd, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
            return JFNK_OK;
        }
        const double alpha = rz / pq;
        JFNK_TRY(axpby<double>(p.delta, pd, alpha, 1.0, N, st));
        JFNK_TRY(axpby<double>(p.tmp64, p.w64, -alpha, 1.0, N, st));
        JFNK_TRY(read_norm(p, p.tmp64, &res, st));
        if (res <= target || !std::isfinite(res)) break;
        JFNK_TRY(apply_mg64<T>(p, o, p.tmp64, p.z64, st));
        double rz_new = 0.0;
        JFNK_TRY(dot2(p, p.tmp64, p.z64, nullptr, nullptr, &rz_new, st));
        const double beta = rz_new / rz;
        rz = rz_new;
        JFNK_TRY(axpby<double>(pd, p.z64, 1.0, beta, N, st));
    }
    return JFNK_OK;
}

static jfnk_status check_status(P& p, cudaStream_t st) {
    int s = 0;
    JFNK_CUDA_TRY(cudaMemcpyAsync(&s, p.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    if (s) {
        set_error("device status word 0x%x (non-finite FD step or eigenvalue estimate)", s);
        return JFNK_ERR_NONFINITE;
    }
    return JFNK_OK;
}

template <typename T>
static jfnk_status solve_T(P& p, const jfnk_options& o, double* u, jfnk_stats* stats, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    const Grid& g = p.lv[p.L].g;
    const long long N = g.size;
    jfnk_stats S;
    memset(&S, 0, sizeof(S));
    for (int l = 0; l <= p.L; ++l) p.nF[l] = p.nFplain[l] = 0;
    long long ci0 = 0;
    JFNK_CUDA_TRY(cudaMemcpyAsync(&ci0, p.coarse_iters, sizeof(long long), cudaMemcpyDeviceToHost, st));
    JFNK_TRY(residual64(p, u, p.F64, p.Au64, st));
    double normF = 0.0;
    JFNK_TRY(read_norm(p, p.F64, &normF, st));
    const double F0 = normF;
    S.res_hist[0] = normF;
    jfnk_status result = JFNK_OK;
    auto converged = [&](double nf) {
        return F0 == 0.0 || nf <= o.rtol_newton * F0 || (o.atol_newton > 0.0 && nf < o.atol_newton);
    };
    int k = 0;
    for (; k < o.max_newton; ++k) {
        if (converged(normF)) break;
        if (!std::isfinite(normF)) {
            result = JFNK_ERR_NONFINITE;
            set_error("non-finite residual norm at Newton step %d", k);
            break;
        }
        // p.Au64 holds A(u) of this iterate (the Newton residual's evaluation)
        JFNK_TRY(mg_setup_T<T>(p, o, u, k, st, p.Au64));
        JFNK_TRY(masked_stat<double>(g, u, 0, p.xstat64, p.red, st));
        const double eta = (o.eta_mode == 1) ? std::fmin(o.eta_max, normF) : std::fmin(o.eta_max, normF / F0);
        JFNK_TRY(axpby<double>(p.rhs64, p.F64, -1.0, 0.0, N, st));
        int its = 0;
        ArnoldiSlope asl;
        if (o.outer == JFNK_OUTER_CG) {
            int negc = 0;
            JFNK_TRY(pcg<T>(p, o, u, eta, its, negc, st));
            S.outer_negcurv += negc;
        } else {
            JFNK_TRY(fgmres<T>(p, o, u, eta, its, st, &asl));
        }
        JFNK_TRY(check_status(p, st));
        S.linear_its += its;
        if (k < JFNK_MAX_HIST) S.lin_hist[k] = its;
        // line search on phi(alpha) = 1/2 ||F(u + alpha delta)||^2
        double alpha = 1.0, normT = 0.0;
        Range rg_ls("line search (Newton step %d)", k);
        if (o.line_search) {
            // phi'(0) = F . (J delta): after a single FGMRES cycle from its Arnoldi
            // relation (rhs = -F = beta v_0, so F . (J Z y) = -beta (Hbar y)_0),
            // otherwise (restarts, CG) from one more FD action
            double slope = 0.0;
            if (asl.cycles == 1) {
                slope = -asl.beta * asl.Hy0;
            } else {
                JFNK_TRY(jv64(p, u, p.Au64, p.delta, p.w64, st));
                JFNK_TRY(multi_dot(p.F64, p.w64, N, N, 1, p.hbuf, p.dot_partials, &p.counters[2], st));
                JFNK_CUDA_TRY(cudaMemcpyAsync(&slope, p.hbuf, sizeof(double), cudaMemcpyDeviceToHost, st));
                JFNK_CUDA_TRY(cudaStreamSynchronize(st));
            }
            const double f0 = 0.5 * normF * normF;
            double prev_a = -1.0, prev_f = 0.0;
            bool ok = false;
            int trials = 0;
            for (int ls = 0; ls < o.ls_max; ++ls) {
                JFNK_TRY(add_scaled(p.utrial, u, alpha, p.delta, N, st));
                JFNK_TRY(residual64(p, p.utrial, p.Ftrial, p.Autrial, st));
                JFNK_TRY(read_norm(p, p.Ftrial, &normT, st));
                trials++;
                const double fn = 0.5 * normT * normT;
                if (std::isfinite(fn) && fn <= f0 + 1e-4 * alpha * slope) {
                    ok = true;
                    break;
                }
                double t;
                if (!std::isfinite(fn)) {
                    // cut the step; the trial is not an interpolation point
                    alpha = 0.1 * alpha;
                    prev_a = -1.0;
                    continue;
                } else if (prev_a < 0.0) {
                    t = -slope * alpha * alpha / (2.0 * (fn - f0 - slope * alpha));
                } else {
                    const double r1 = fn - f0 - slope * alpha;
                    const double r2 = prev_f - f0 - slope * prev_a;
                    const double A = (r1 / (alpha * alpha) - r2 / (prev_a * prev_a)) / (alpha - prev_a);
                    const double B = (-prev_a * r1 / (alpha * alpha) + alpha * r2 / (prev_a * prev_a)) / (alpha - prev_a);
                    if (A == 0.0) {
                        t = -slope / (2.0 * B);
                    } else {
                        const double disc = B * B - 3.0 * A * slope;
                        t = disc >= 0.0 ? (-B + std::sqrt(disc)) / (3.0 * A) : 0.5 * alpha;
                    }
                }
                t = std::fmin(std::fmax(t, 0.1 * alpha), 0.5 * alpha);
                prev_a = alpha;
                prev_f = fn;
                alpha = t;
            }
            if (k < JFNK_MAX_HIST) S.ls_hist[k] = trials;
            if (!ok) {
                // no sufficient decrease: the step is not taken and the solve
                // stops at the last accepted iterate (Dennis & Schnabel, Sec. 6.3)
                result = JFNK_ERR_LINESEARCH;
                if (k + 1 < JFNK_MAX_HIST) S.res_hist[k + 1] = normF;
                if (k < JFNK_MAX_HIST) S.alpha_hist[k] = 0.0;
                set_error("line search found no sufficient decrease in %d trials at Newton step %d", trials, k);
                k++;
                break;
            }
        } else {
            JFNK_TRY(add_scaled(p.utrial, u, 1.0, p.delta, N, st));
            JFNK_TRY(residual64(p, p.utrial, p.Ftrial, p.Autrial, st));
            JFNK_TRY(read_norm(p, p.Ftrial, &normT, st));
            if (k < JFNK_MAX_HIST) S.ls_hist[k] = 1;
        }
        JFNK_CUDA_TRY(cudaMemcpyAsync(u, p.utrial, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        std::swap(p.F64, p.Ftrial);
        std::swap(p.Au64, p.Autrial);
        normF = normT;
        if (k + 1 < JFNK_MAX_HIST) S.res_hist[k + 1] = normF;
        if (k < JFNK_MAX_HIST) S.alpha_hist[k] = alpha;
    }
    S.newton_its = k;
    S.converged = converged(normF) ? 1 : 0;
    if (result == JFNK_OK && !S.converged) {
        result = JFNK_ERR_NOT_CONVERGED;
        set_error("Newton did not reach the tolerance in %d steps", k);
    }
    long long ci1 = 0;
    JFNK_CUDA_TRY(cudaMemcpyAsync(&ci1, p.coarse_iters, sizeof(long long), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    p.nF[0] += ci1 - ci0;
    double ge = 0.0;
    for (int l = 0; l <= p.L && l < JFNK_MAX_LEVELS; ++l) {
        S.nF[l] = p.nF[l];
        S.nJv[l] = p.nF[l] - p.nFplain[l];
        ge += std::pow(2.0, -(double)p.d * (p.L - l)) * (double)p.nF[l];
        double lam = 0.0;
        if (l >= 1) {
            JFNK_CUDA_TRY(cudaMemcpy(&lam, p.lv[l].lam, sizeof(double), cudaMemcpyDeviceToHost));
        }
        S.lambda_max[l] = lam;
    }
    S.ge = ge;
    if (p.lb) {
        int hs[4] = {0, 0, 0, 0};
        JFNK_CUDA_TRY(cudaMemcpy(hs, p.lb, sizeof(hs), cudaMemcpyDeviceToHost));
        S.coarse_shifts = hs[2];
        S.coarse_negcurv = hs[3];
    }
    S.status = result;
    S.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    return result;
}

static jfnk_status check_opts(const P& p, const jfnk_options* o) {
    if (!o) return JFNK_ERR_INVALID_ARG;
    if (o->restart < 1 || o->restart > JFNK_MAX_RESTART || o->cheb_degree < 1 ||
        o->cheb_degree > kMaxChebDegree || o->nu_pre < 0 || o->nu_post < 0 || o->power_iters < 1 ||
        !(o->cheb_hi > o->cheb_lo) || !(o->cheb_lo > 0.0) || (o->pc_dtype != JFNK_F32 && o->pc_dtype != JFNK_F64) ||
        (o->eps_mode_pc != JFNK_EPS_PAPER && o->eps_mode_pc != JFNK_EPS_FP32) || o->max_linear < 1 ||
        (o->outer != JFNK_OUTER_FGMRES && o->outer != JFNK_OUTER_CG) ||
        (o->coarse_method != JFNK_COARSE_GMRES && o->coarse_method != JFNK_COARSE_CGQN) ||
        (o->coarse_method == JFNK_COARSE_CGQN && (o->lbfgs_pairs < 1 || o->lbfgs_pairs > kMaxLbfgsPairs ||
                                                  !(o->shift_gamma > 1.0)))) {
        set_error("invalid options");
        return JFNK_ERR_INVALID_ARG;
    }
    return JFNK_OK;
}

static jfnk_status need_solver(const P* p, const jfnk_options* o) {
    if (!p || !p->bound) {
        set_error("no workspace attached");
        return JFNK_ERR_WORKSPACE;
    }
    JFNK_TRY(check_opts(*p, o));
    if (!p->has_solver || o->pc_dtype != p->pc || o->restart > p->m) {
        set_error("workspace was laid out for other options (pc dtype %d, restart %d)", p->pc, p->m);
        return JFNK_ERR_WORKSPACE;
    }
    const int cm = o->coarse_maxit > 0 ? o->coarse_maxit : (int)p->lv[0].g.interior();
    if (cm > p->coarse_maxit) {
        set_error("coarse_maxit exceeds the workspace layout");
        return JFNK_ERR_WORKSPACE;
    }
    return JFNK_OK;
}

}  // namespace jfnk

// ===========================================================================
// C ABI
// ===========================================================================
using namespace jfnk;

// The exported functions below were declared extern "C" in jfnk.h, so their
// definitions keep C linkage.

const char* jfnk_last_error(void) { return g_err.c_str(); }

jfnk_status jfnk_debug_bounds(int* enabled, unsigned int* line, int reset) {
    using namespace jfnk;
    int on = 0;
#ifdef JFNK_DEBUG_BOUNDS
    on = 1;
#endif
    if (enabled) *enabled = on;
    unsigned int first = 0;
    for (const auto& e : bounds_registry()) {
        const unsigned int v = e.reader(reset);
        if (v == 0xffffffffu) {
            set_error("jfnk_debug_bounds: reading the record of %s failed", e.file);
            return JFNK_ERR_CUDA;
        }
        if (v && !first) {
            first = v;
            set_error("index out of range at %s:%u", e.file, v);
        }
    }
    if (line) *line = first;
    return JFNK_OK;
}

long long jfnk_kernel_launches(int reset) {
    long long v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

void jfnk_default_options(jfnk_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->nu_pre = 3;
    o->nu_post = 3;
    o->cheb_degree = 3;
    o->cheb_lo = 0.1;
    o->cheb_hi = 1.1;
    o->power_iters = 10;
    o->power_tol = 0.0;
    o->restart = 30;
    o->max_linear = 300;
    o->rtol_newton = 1e-10;
    o->atol_newton = 0.0;
    o->eta_mode = 0;
    o->eta_max = 0.5;
    o->coarse_tol = 1e-12;
    o->coarse_tol_mode = 0;
    o->coarse_maxit = 0;
    o->pc_dtype = JFNK_F64;
    o->eps_mode_pc = JFNK_EPS_PAPER;
    o->max_newton = 50;
    o->line_search = 1;
    o->ls_max = 10;
    o->seed = 0;
    o->use_graph = 1;
    o->outer = JFNK_OUTER_FGMRES;
    o->coarse_method = JFNK_COARSE_GMRES;
    o->lbfgs_pairs = 20;
    o->shift_gamma = 5.0;
}

void jfnk_paper_options(jfnk_options* o) {
    if (!o) return;
    jfnk_default_options(o);
    o->nu_pre = 1;
    o->nu_post = 1;
    o->cheb_degree = 5;
    o->cheb_lo = 0.06;
    o->cheb_hi = 1.2;
    o->power_iters = 30;
    o->power_tol = 1e-2;
    o->rtol_newton = 0.0;
    o->atol_newton = 1e-6;
    o->eta_mode = 1;
    o->outer = JFNK_OUTER_CG;
    o->coarse_method = JFNK_COARSE_CGQN;
    o->lbfgs_pairs = 20;
    o->shift_gamma = 5.0;
}

jfnk_status jfnk_problem_create(const jfnk_problem_desc* desc, jfnk_problem** out) {
    if (!desc || !out) {
        set_error("null argument");
        return JFNK_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (desc->kind < JFNK_BRATU2D || desc->kind > JFNK_BEAM3D) {
        set_error("unknown problem kind %d", desc->kind);
        return JFNK_ERR_INVALID_ARG;
    }
    if (desc->levels < 1 || desc->levels > JFNK_MAX_LEVELS || desc->n_elem < 1) {
        set_error("invalid levels %d / n_elem %d", desc->levels, desc->n_elem);
        return JFNK_ERR_INVALID_ARG;
    }
    const int L = desc->levels - 1;
    const int min_coarse = desc->kind == JFNK_BEAM3D ? 1 : 2;
    if ((desc->n_elem >> L) < min_coarse || ((desc->n_elem >> L) << L) != desc->n_elem) {
        set_error("n_elem %d is not divisible into %d levels with >= %d coarse elements", desc->n_elem, desc->levels,
                  min_coarse);
        return JFNK_ERR_INVALID_ARG;
    }
    if (desc->kind == JFNK_NDK3D && !desc->kappa) {
        set_error("NDK3D needs kappa");
        return JFNK_ERR_INVALID_ARG;
    }
    const int d = (desc->kind == JFNK_BRATU2D || desc->kind == JFNK_MINSURF2D) ? 2 : 3;
    const long long len_mult = desc->kind == JFNK_BEAM3D ? 30 : 1;  // 10x the nodes, 3 components
    if (d == 3 && (long long)(desc->n_elem + 1) * (desc->n_elem + 1) * (desc->n_elem + 1) * len_mult > (1LL << 31)) {
        set_error("grid too large");
        return JFNK_ERR_INVALID_ARG;
    }
    P* p = new P();
    p->desc = *desc;
    p->d = d;
    p->L = L;
    p->n = desc->n_elem;
    cudaGetDevice(&p->device);
    p->lv.resize(L + 1);
    for (int l = 0; l <= L; ++l) {
        const int nl = desc->n_elem >> (L - l);
        p->lv[l].g = desc->kind == JFNK_BEAM3D ? Grid::make_beam(nl) : Grid::make(d, nl);
        p->lv[l].h = 1.0 / (double)(desc->n_elem >> (L - l));
        p->lv[l].pv_valid = false;
    }
    *out = p;
    return JFNK_OK;
}

jfnk_status jfnk_problem_destroy(jfnk_problem* p) {
    if (p) {
        if (p->vgraph) cudaGraphExecDestroy(p->vgraph);
        if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    }
    delete p;
    return JFNK_OK;
}

jfnk_status jfnk_workspace_size(const jfnk_problem* p, const jfnk_options* opts, size_t* bytes) {
    if (!p || !bytes) {
        set_error("null argument");
        return JFNK_ERR_INVALID_ARG;
    }
    if (opts) JFNK_TRY(check_opts(*p, opts));
    P tmp = *p;
    *bytes = plan(tmp, nullptr, opts) + 256;
    return JFNK_OK;
}

// 1D tables of the manufactured load (see mms_load in transfer.cu), 3-point
// Gauss rule per element, computed on the host in FP64.
static void mms_tables(int n, std::vector<double>& tab) {
    const int np = n + 1;
    tab.assign(3 * (size_t)np, 0.0);
    const double h = 1.0 / n;
    const double gp[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    const double pi = 3.14159265358979323846;
    for (int e = 0; e < n; ++e) {
        for (int q = 0; q < 3; ++q) {
            const double x = (e + gp[q]) * h;
            const double s = std::sin(pi * x), c = std::cos(pi * x);
            const double w = gw[q] * h;
            const double phi[2] = {1.0 - gp[q], gp[q]};
            for (int a = 0; a < 2; ++a) {
                tab[e + a] += w * s * phi[a];
                tab[np + e + a] += w * s * s * s * phi[a];
                tab[2 * np + e + a] += w * s * c * c * phi[a];
            }
        }
    }
}

jfnk_status jfnk_set_workspace(jfnk_problem* p, const jfnk_options* opts, void* dev_ptr, size_t bytes, void* stream) {
    if (!p || !dev_ptr) {
        set_error("null argument");
        return JFNK_ERR_INVALID_ARG;
    }
    if (opts) JFNK_TRY(check_opts(*p, opts));
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)(((uintptr_t)dev_ptr + 255) & ~uintptr_t(255));
    const size_t need = plan(*p, nullptr, opts);
    if ((size_t)(base - (char*)dev_ptr) + need > bytes) {
        set_error("workspace too small: %zu bytes needed", need + 256);
        return JFNK_ERR_WORKSPACE;
    }
    plan(*p, base, opts);
    if (p->vgraph) {  // the captured cycle refers to the previous workspace
        cudaGraphExecDestroy(p->vgraph);
        p->vgraph = nullptr;
    }
    p->ws = base;
    p->ws_bytes = need;
    p->has_solver = opts != nullptr;
    p->pc = opts ? opts->pc_dtype : JFNK_F64;
    p->m = opts ? opts->restart : 0;
    p->coarse_maxit = opts ? (opts->coarse_maxit > 0 ? opts->coarse_maxit : (int)p->lv[0].g.interior()) : 0;
    if (p->has_solver && (p->coarse_maxit > JFNK_COARSE_MAX_IT || p->lv[0].g.size > JFNK_COARSE_MAX_NODES)) {
        set_error("coarse level too large for the single-CTA solver: %lld nodes, %d iterations (limits %d, %d)",
                  p->lv[0].g.size, p->coarse_maxit, JFNK_COARSE_MAX_NODES, JFNK_COARSE_MAX_IT);
        return JFNK_ERR_INVALID_ARG;
    }
    JFNK_CUDA_TRY(cudaMemsetAsync(base, 0, need, st));
    for (auto& L : p->lv) L.pv_valid = false;
    // coefficient hierarchy (NDK): finest copied, coarser levels averaged
    if (p->desc.kind == JFNK_NDK3D) {
        Level& Lf = p->lv[p->L];
        const size_t ne = (size_t)Lf.g.n * Lf.g.n * Lf.g.n;
        JFNK_CUDA_TRY(cudaMemcpyAsync(Lf.kappa64, p->desc.kappa, ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (int l = p->L; l >= 1; --l)
            JFNK_TRY(coarsen_kappa(p->lv[l - 1].g.n, p->lv[l].kappa64, p->lv[l - 1].kappa64, st));
        for (int l = 0; l <= p->L; ++l) {
            const long long nel = (long long)p->lv[l].g.n * p->lv[l].g.n * p->lv[l].g.n;
            JFNK_TRY((cast_copy<float, double>(p->lv[l].kappa32, p->lv[l].kappa64, nel, st)));
        }
    }
    if (p->desc.kind == JFNK_ND3D) {
        const Grid& g = p->lv[p->L].g;
        if (p->desc.load) {
            JFNK_CUDA_TRY(cudaMemcpyAsync(p->load64, p->desc.load, g.size * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            std::vector<double> tab;
            mms_tables(g.n, tab);
            JFNK_CUDA_TRY(cudaMemcpyAsync(p->mms_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            JFNK_TRY(mms_load(g, p->mms_tab, p->load64, st));
            JFNK_CUDA_TRY(cudaStreamSynchronize(st));  // tab is host memory
        }
        JFNK_TRY((cast_copy<float, double>(p->load32, p->load64, g.size, st)));
    }
    p->bound = true;
    return JFNK_OK;
}

static jfnk_status check_level(const jfnk_problem* p, int level, int dtype) {
    if (!p || !p->bound) {
        set_error("no workspace attached");
        return JFNK_ERR_WORKSPACE;
    }
    if (level < 0 || level > p->L || (dtype != JFNK_F32 && dtype != JFNK_F64)) {
        set_error("invalid level %d or dtype %d", level, dtype);
        return JFNK_ERR_INVALID_ARG;
    }
    return JFNK_OK;
}

template <typename T>
static jfnk_status residual_T(P* p, int level, const T* u, T* F, cudaStream_t st);
template <>
jfnk_status residual_T<double>(P* p, int level, const double* u, double* F, cudaStream_t st) {
    StencilArgs<double> a = base_args<double>(*p, level);
    a.u = u;
    a.out = F;
    if (level == p->L) {
        a.load = p->load64;
        a.load_const = (p->desc.kind == JFNK_NDK3D) ? std::pow(p->lv[level].h, 3) : 0.0;
    }
    return launch_stencil<double>(prob_of(*p), Mode::F, a, st);
}
template <>
jfnk_status residual_T<float>(P* p, int level, const float* u, float* F, cudaStream_t st) {
    StencilArgs<float> a = base_args<float>(*p, level);
    a.u = u;
    a.out = F;
    if (level == p->L) {
        a.load = p->load32;
        a.load_const = (p->desc.kind == JFNK_NDK3D) ? std::pow(p->lv[level].h, 3) : 0.0;
    }
    return launch_stencil<float>(prob_of(*p), Mode::F, a, st);
}

jfnk_status jfnk_residual(jfnk_problem* p, int level, int dtype, const void* u, void* F, void* stream) {
    JFNK_TRY(check_level(p, level, dtype));
    if (!u || !F) {
        set_error("null vector");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == JFNK_F64) return residual_T<double>(p, level, (const double*)u, (double*)F, st);
    return residual_T<float>(p, level, (const float*)u, (float*)F, st);
}

template <typename T>
static jfnk_status jvp_T(P* p, int level, const T* u, const T* Fu, const T* v, T* Jv, double eps, int eps_mode,
                         cudaStream_t st) {
    Level& L = p->lv[level];
    if (eps > 0.0) {
        JFNK_TRY(set_eps(L.eps_aux, eps, st));
    } else {
        EpsParams ep = eps_params(*p, level, eps_mode);
        JFNK_TRY(masked_stat<T>(L.g, u, eps_mode == JFNK_EPS_PAPER ? 0 : 1, const_cast<double*>(ep.xstat), p->red, st));
        JFNK_TRY(norm_to_eps<T>(L.g, v, ep, L.eps_aux, nullptr, p->red, st));
    }
    StencilArgs<T> a = base_args<T>(*p, level);
    a.u = u;
    a.v = v;
    a.eps = L.eps_aux;
    a.Au = Fu;  // F(u): the same load is removed from A(u + eps v) below
    a.out = Jv;
    if (level == p->L) {
        a.load = load_of<T>(*p);
        a.load_const = (p->desc.kind == JFNK_NDK3D) ? std::pow(L.h, 3) : 0.0;
    }
    return launch_stencil<T>(prob_of(*p), Mode::JV, a, st);
}

jfnk_status jfnk_jvp(jfnk_problem* p, int level, int dtype, const void* u, const void* Fu, const void* v, void* Jv,
                     double eps, int eps_mode, void* stream) {
    JFNK_TRY(check_level(p, level, dtype));
    if (!u || !Fu || !v || !Jv || (eps_mode != JFNK_EPS_PAPER && eps_mode != JFNK_EPS_FP32)) {
        set_error("invalid jvp arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == JFNK_F64)
        return jvp_T<double>(p, level, (const double*)u, (const double*)Fu, (const double*)v, (double*)Jv, eps,
                             eps_mode, st);
    return jvp_T<float>(p, level, (const float*)u, (const float*)Fu, (const float*)v, (float*)Jv, eps, eps_mode, st);
}

jfnk_status jfnk_mg_setup(jfnk_problem* p, const jfnk_options* opts, const double* u, int newton_step, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (!u) return JFNK_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->pc == JFNK_F32) return mg_setup_T<float>(*p, *opts, u, newton_step, st);
    return mg_setup_T<double>(*p, *opts, u, newton_step, st);
}

template <typename T>
static jfnk_status vcycle_api(P& p, const jfnk_options& o, const double* b, double* s, cudaStream_t st) {
    Level& Lf = p.lv[p.L];
    JFNK_TRY((cast_copy<T, double>(as<T>(Lf.b), b, Lf.g.size, st)));
    T* sT = as<T>(p.Z);  // first Krylov slot as the output buffer
    JFNK_TRY(vcycle<T>(p, o, p.L, as<T>(Lf.b), sT, st));
    JFNK_TRY((cast_copy<double, T>(s, sT, Lf.g.size, st)));
    return JFNK_OK;
}

jfnk_status jfnk_mg_vcycle(jfnk_problem* p, const jfnk_options* opts, const double* b, double* s, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (!b || !s) return JFNK_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->pc == JFNK_F32) return vcycle_api<float>(*p, *opts, b, s, st);
    return vcycle_api<double>(*p, *opts, b, s, st);
}

jfnk_status jfnk_solve(jfnk_problem* p, const jfnk_options* opts, double* u_inout, jfnk_stats* stats, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (!u_inout) return JFNK_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->pc == JFNK_F32) return solve_T<float>(*p, *opts, u_inout, stats, st);
    return solve_T<double>(*p, *opts, u_inout, stats, st);
}


// ---- building blocks exposed one by one -----------------------------------

jfnk_status jfnk_transfer(jfnk_problem* p, int op, int level, int dtype, const void* in, void* out, void* stream) {
    JFNK_TRY(check_level(p, level, dtype));
    if (level < 1 || !in || !out || op < JFNK_RESTRICT || op > JFNK_PROJECT) {
        set_error("invalid transfer arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const Grid& gf = p->lv[level].g;
    const Grid& gc = p->lv[level - 1].g;
    if (dtype == JFNK_F64) {
        if (op == JFNK_PROLONG_ADD) return prolong_add<double>(gc, gf, (const double*)in, (double*)out, st);
        return restrict_to<double>(gf, gc, (const double*)in, (double*)out, op == JFNK_PROJECT, st);
    }
    if (op == JFNK_PROLONG_ADD) return prolong_add<float>(gc, gf, (const float*)in, (float*)out, st);
    return restrict_to<float>(gf, gc, (const float*)in, (float*)out, op == JFNK_PROJECT, st);
}

jfnk_status jfnk_smooth(jfnk_problem* p, const jfnk_options* opts, int level, const void* b, void* s, int nu,
                        int s_is_zero, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (level < 1 || level > p->L || !b || !s || nu < 0) {
        set_error("invalid smooth arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Level& L = p->lv[level];
    if (p->pc == JFNK_F32) {
        if (!s_is_zero) JFNK_TRY(norm_to_eps<float>(L.g, (const float*)s, eps_params(*p, level, opts->eps_mode_pc), L.eps_s, nullptr, p->red, st));
        return smooth<float>(*p, *opts, level, (const float*)b, (float*)s, nu, s_is_zero != 0, st);
    }
    if (!s_is_zero) JFNK_TRY(norm_to_eps<double>(L.g, (const double*)s, eps_params(*p, level, opts->eps_mode_pc), L.eps_s, nullptr, p->red, st));
    return smooth<double>(*p, *opts, level, (const double*)b, (double*)s, nu, s_is_zero != 0, st);
}

jfnk_status jfnk_coarse_solve(jfnk_problem* p, const jfnk_options* opts, const void* b, void* s, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (!b || !s) return JFNK_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->pc == JFNK_F32) return coarse_solve<float>(*p, *opts, (const float*)b, (float*)s, st);
    return coarse_solve<double>(*p, *opts, (const double*)b, (double*)s, st);
}

jfnk_status jfnk_level_info(jfnk_problem* p, int level, double* lambda_max, double* xstat_l1, double* xstat_l2,
                            void* stream) {
    if (!p || !p->bound || level < 0 || level > p->L) {
        set_error("invalid level_info arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Level& L = p->lv[level];
    double v[3] = {0, 0, 0};
    JFNK_CUDA_TRY(cudaMemcpyAsync(&v[0], L.lam, sizeof(double), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(&v[1], L.xstat_paper, sizeof(double), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(&v[2], L.xstat_fp32, sizeof(double), cudaMemcpyDeviceToHost, st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    if (lambda_max) *lambda_max = v[0];
    if (xstat_l1) *xstat_l1 = v[1];
    if (xstat_l2) *xstat_l2 = v[2];
    return JFNK_OK;
}

jfnk_status jfnk_level_vector(jfnk_problem* p, int level, int which, void* out, void* stream) {
    if (!p || !p->bound || !p->has_solver || level < 0 || level > p->L || which < 0 || which > 2 || !out) {
        set_error("invalid level_vector arguments");
        return JFNK_ERR_INVALID_ARG;
    }
    Level& L = p->lv[level];
    const void* src = which == 0 ? L.x : which == 1 ? L.Ax : L.pv;
    const size_t esz = p->pc == JFNK_F32 ? 4 : 8;
    JFNK_CUDA_TRY(cudaMemcpyAsync(out, src, esz * L.g.size, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return JFNK_OK;
}

// ---- adjoint (vector-Jacobian products, adjoint solve) --------------------

template <typename T>
static jfnk_status vjp_T(P* p, int level, const T* u, const T* w, T* JTw, T* dk, cudaStream_t st) {
    StencilArgs<T> a = base_args<T>(*p, level);
    a.u = u;
    a.v = w;
    a.out = JTw;
    a.dkout = dk;
    a.dk_scale = (T)(1.5 * p->lv[level].h);  // (dF/dkappa_e)^T w = (3h/2) x element sum
    return launch_vjp<T>(prob_of(*p), Mode::JV, a, st);
}

jfnk_status jfnk_vjp(jfnk_problem* p, int level, int dtype, const void* u, const void* w, void* JTw,
                     void* dFdkappa_w, void* stream) {
    JFNK_TRY(check_level(p, level, dtype));
    if (!u || !w || !JTw || p->d == 2 || p->desc.kind == JFNK_BEAM3D) {
        set_error("jfnk_vjp: null vector or 2D problem (Bratu's J is symmetric: use jfnk_jvp)");
        return JFNK_ERR_INVALID_ARG;
    }
    if (dFdkappa_w && p->desc.kind != JFNK_NDK3D) {
        set_error("dF/dkappa exists for the coefficient problem only");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == JFNK_F64)
        return vjp_T<double>(p, level, (const double*)u, (const double*)w, (double*)JTw, (double*)dFdkappa_w, st);
    return vjp_T<float>(p, level, (const float*)u, (const float*)w, (float*)JTw, (float*)dFdkappa_w, st);
}

jfnk_status jfnk_set_kappa(jfnk_problem* p, const double* kappa, void* stream) {
    if (!p || !p->bound || !kappa || p->desc.kind != JFNK_NDK3D) {
        set_error("jfnk_set_kappa: needs a bound coefficient problem and a kappa pointer");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Level& Lf = p->lv[p->L];
    const size_t ne = (size_t)Lf.g.n * Lf.g.n * Lf.g.n;
    JFNK_CUDA_TRY(cudaMemcpyAsync(Lf.kappa64, kappa, ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int l = p->L; l >= 1; --l) JFNK_TRY(coarsen_kappa(p->lv[l - 1].g.n, p->lv[l].kappa64, p->lv[l - 1].kappa64, st));
    for (int l = 0; l <= p->L; ++l) {
        const long long nel = (long long)p->lv[l].g.n * p->lv[l].g.n * p->lv[l].g.n;
        JFNK_TRY((cast_copy<float, double>(p->lv[l].kappa32, p->lv[l].kappa64, nel, st)));
    }
    for (auto& L : p->lv) L.pv_valid = false;
    return JFNK_OK;
}

template <typename T>
static jfnk_status adjoint_T(P& p, const jfnk_options& o, const double* u, const double* g, double* lambda,
                             double* grad_kappa, double rtol, jfnk_stats* stats, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    struct AdjGuard {
        P& q;
        explicit AdjGuard(P& qq) : q(qq) { q.adj = true; }
        ~AdjGuard() { q.adj = false; }
    } guard(p);
    for (int l = 0; l <= p.L; ++l) p.nF[l] = p.nFplain[l] = 0;
    const Grid& gf = p.lv[p.L].g;
    // hierarchy at u; the power method now estimates lambda of J^T (same spectrum as J)
    JFNK_TRY(mg_setup_T<T>(p, o, u, 0, st));
    JFNK_TRY((cast_scale_interior<double, double>(p.rhs64, g, 1.0, gf, st)));
    int its = 0;
    JFNK_TRY(fgmres<T>(p, o, u, rtol, its, st));
    JFNK_TRY(check_status(p, st));
    JFNK_CUDA_TRY(cudaMemcpyAsync(lambda, p.delta, sizeof(double) * gf.size, cudaMemcpyDeviceToDevice, st));
    if (grad_kappa) {
        // grad_kappa = -(dF/dkappa)^T lambda  (F(u(kappa), kappa) = 0)
        StencilArgs<double> a = base_args<double>(p, p.L);
        a.u = u;
        a.v = p.delta;
        a.out = p.w64;
        a.dkout = grad_kappa;
        a.dk_scale = -1.5 * p.lv[p.L].h;
        JFNK_TRY(launch_vjp<double>(prob_of(p), Mode::JV, a, st));
    }
    JFNK_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats) {
        jfnk_stats S;
        memset(&S, 0, sizeof(S));
        S.linear_its = its;
        S.lin_hist[0] = its;
        S.converged = 1;
        double ge = 0.0;
        for (int l = 0; l <= p.L && l < JFNK_MAX_LEVELS; ++l) {
            S.nF[l] = p.nF[l];
            S.nJv[l] = p.nF[l] - p.nFplain[l];
            ge += std::pow(2.0, -(double)p.d * (p.L - l)) * (double)p.nF[l];
            if (l >= 1) JFNK_CUDA_TRY(cudaMemcpy(&S.lambda_max[l], p.lv[l].lam, sizeof(double), cudaMemcpyDeviceToHost));
        }
        S.ge = ge;
        S.status = JFNK_OK;
        S.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *stats = S;
    }
    return JFNK_OK;
}

jfnk_status jfnk_adjoint_solve(jfnk_problem* p, const jfnk_options* opts, const double* u, const double* g,
                               double* lambda, double* grad_kappa, double rtol, jfnk_stats* stats, void* stream) {
    JFNK_TRY(need_solver(p, opts));
    if (!u || !g || !lambda || p->d == 2 || p->desc.kind == JFNK_BEAM3D || !(rtol > 0.0)) {
        set_error("jfnk_adjoint_solve: invalid arguments (3D diffusion problems only, rtol > 0)");
        return JFNK_ERR_INVALID_ARG;
    }
    if (grad_kappa && p->desc.kind != JFNK_NDK3D) {
        set_error("grad_kappa exists for the coefficient problem only");
        return JFNK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->pc == JFNK_F32) return adjoint_T<float>(*p, *opts, u, g, lambda, grad_kappa, rtol, stats, st);
    return adjoint_T<double>(*p, *opts, u, g, lambda, grad_kappa, rtol, stats, st);
}

#include "batch_solver.cuh"
