// Batched inexact-Newton / FGMRES / multigrid solve of independent 2D Bratu
// instances of uneven sizes (included once, at the end of solver.cu).
//
// Every instance keeps its own problem object and workspace; the instances
// advance in lock step and every device operation is ONE launch over all
// instances it applies to: the level operations of the V-cycle (Chebyshev
// steps, b - J s, restriction, prolongation, norms) over the instances that
// have that level (all hierarchies end at the same 8 x 8 coarse grid, so the
// levels align from the coarse end), the coarse GMRES with one CTA per
// instance, and the FGMRES / Newton vector operations over the instances
// still iterating.  Per instance the sequence of operations and the
// arithmetic are those of jfnk_solve.  The V-cycle's per-instance operands
// are assembled once into a descriptor program in device memory and replayed
// (from a CUDA graph when opts->use_graph is set); it is rebuilt only when the
// set of instances still iterating changes.

namespace jfnk {

// Device staging of descriptor arrays in the lead problem's workspace.
struct Arena {
    char* dev = nullptr;
    size_t cap = 0, off = 0;
    std::vector<char> host;
    bool replay = false;  // recompute offsets only (program replay)
    void reset() {
        off = 0;
        host.clear();
        replay = false;
    }
    template <class D>
    D* put(const std::vector<D>& v) {
        const size_t bytes = ((v.size() * sizeof(D)) + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        D* ptr = reinterpret_cast<D*>(dev + off);
        if (!replay) {
            host.resize(off + bytes);
            if (!v.empty()) memcpy(host.data() + off, v.data(), v.size() * sizeof(D));
        }
        off += bytes;
        return ptr;
    }
};

// Tiling of the batched 2D kernel: threads per CTA, target CTA count of a
// launch (sets the row-chunk length), persistent grid size (0: one CTA per tile).
struct TileCfg {
    int bx = 160;
    int target = 608;
    int grid = 0;
};

struct BCtx {
    TileCfg tile[2];  // [0] FP32, [1] FP64 launches
    std::vector<P*> ps;
    std::vector<double*> u;
    int B = 0;
    const jfnk_options* o = nullptr;
    cudaStream_t st = nullptr;
    P* lead = nullptr;
    Arena prog, dyn;
    double* res = nullptr;  // per-instance results, kResStride doubles each
    bool dry = false;       // program build pass: descriptors only, no launches
    bool immediate = true;  // dyn arena: upload each op's descriptors at once
    // cached V-cycle program
    std::vector<int> prog_set;
    cudaGraphExec_t graph = nullptr;
    ~BCtx() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};
constexpr int kResStride = 2 * JFNK_MAX_RESTART + 16;

static std::vector<int> levels_of(const BCtx& b) {
    std::vector<int> L(b.B);
    for (int i = 0; i < b.B; ++i) L[i] = b.ps[i]->L;
    return L;
}

template <class D>
static D* stage(BCtx& b, Arena& A, const std::vector<D>& v, jfnk_status& err) {
    if (&A == &b.dyn && b.immediate) {
        const size_t bytes = ((v.size() * sizeof(D)) + 255) & ~size_t(255);
        if (A.off + bytes > A.cap) A.off = 0;  // ring: earlier uses are stream-ordered before this copy
        D* ptr = reinterpret_cast<D*>(A.dev + A.off);
        A.off += bytes;
        cudaError_t e = cudaMemcpyAsync(ptr, v.data(), v.size() * sizeof(D), cudaMemcpyHostToDevice, b.st);
        if (e != cudaSuccess) {
            set_error("descriptor upload: %s", cudaGetErrorString(e));
            err = JFNK_ERR_CUDA;
        }
        return ptr;
    }
    D* ptr = A.put(v);
    if (!ptr) {
        set_error("batched descriptor program exceeds its staging area");
        err = JFNK_ERR_WORKSPACE;
    }
    return ptr;
}

static std::vector<BItem> vec_items(const std::vector<long long>& sizes, int cap = 32) {
    std::vector<BItem> it;
    for (int k = 0; k < (int)sizes.size(); ++k) {
        long long nb = (sizes[k] + 255) / 256;
        nb = std::max(1LL, std::min<long long>(nb, cap));
        for (int q = 0; q < nb; ++q) it.push_back(BItem{k, q, (int)nb, 0});
    }
    return it;
}

// tiles of the 2D kernel for grids g[k]: row segments of <= bx-1 nodes, row
// chunks sized so that the launch has about `target` tiles
constexpr int kBatchBX = 160;
static std::vector<BTile> tiles_for(const std::vector<Grid>& gs, int bx = kBatchBX, int target = 608) {
    long long rows = 0;
    for (const Grid& g : gs) rows += (long long)g.ny * ((g.nx + bx - 2) / (bx - 1));
    const int yc = (int)std::max(4LL, (rows + target - 1) / target);
    std::vector<BTile> t;
    for (int k = 0; k < (int)gs.size(); ++k) {
        const Grid& g = gs[k];
        const int segs = (g.nx + bx - 2) / (bx - 1);
        const int txo = (g.nx + segs - 1) / segs;
        const int ch = (g.ny + yc - 1) / yc;
        const int nblk = segs * ch;
        int bid = 0;
        for (int c = 0; c < ch; ++c)
            for (int sg = 0; sg < segs; ++sg)
                t.push_back(BTile{k, sg * txo, c * yc, std::min(c * yc + yc, g.ny), txo, bid++, nblk, 0});
    }
    return t;
}

template <typename T>
static jfnk_status bstencil(BCtx& b, Arena& A, Mode m, const std::vector<int>& S, int lvl_from_coarse,
                            const std::vector<StencilArgs<T>>& args) {
    if (S.empty()) return JFNK_OK;
    std::vector<Grid> gs;
    for (int i : S) gs.push_back(b.ps[i]->lv[lvl_from_coarse].g);
    jfnk_status err = JFNK_OK;
    const TileCfg& tc = b.tile[sizeof(T) == 8 ? 1 : 0];
    const std::vector<BTile> tiles = tiles_for(gs, tc.bx, tc.target);
    const StencilArgs<T>* da = stage(b, A, args, err);
    const BTile* dt = stage(b, A, tiles, err);
    if (err != JFNK_OK) return err;
    if (b.dry) return JFNK_OK;
    return launch_stencil2d_batched<T>(m, da, dt, (int)tiles.size(), tc.bx, b.st, tc.grid);
}

template <typename T>
static jfnk_status bvec(BCtx& b, Arena& A, BOp op, const std::vector<BVec>& d, const std::vector<long long>& sizes) {
    if (d.empty()) return JFNK_OK;
    jfnk_status err = JFNK_OK;
    const std::vector<BItem> items = vec_items(sizes);
    const BVec* dd = stage(b, A, d, err);
    const BItem* di = stage(b, A, items, err);
    if (err != JFNK_OK) return err;
    if (b.dry) return JFNK_OK;
    return launch_bvec<T>(op, dd, di, (int)items.size(), b.st);
}

static jfnk_status bscalar(BCtx& b, Arena& A, BScalar op, const std::vector<BScal>& d) {
    if (d.empty()) return JFNK_OK;
    jfnk_status err = JFNK_OK;
    const BScal* dd = stage(b, A, d, err);
    if (err != JFNK_OK) return err;
    if (b.dry) return JFNK_OK;
    return launch_bscalar(op, dd, (int)d.size(), b.st);
}

static BVec bv0() {
    BVec v;
    memset(&v, 0, sizeof(v));
    return v;
}

// ---------------------------------------------------------------------------
// Chebyshev smoothing at level l (from the coarse end) of instances S
template <typename T>
static jfnk_status bsmooth(BCtx& b, Arena& A, int l, const std::vector<int>& S, int nu, bool s_zero) {
    const jfnk_options& o = *b.o;
    const int k = o.cheb_degree;
    std::vector<long long> sizes;
    for (int i : S) sizes.push_back(b.ps[i]->lv[l].g.size);
    // per-instance ping-pong state (host side, same sequence as smooth())
    std::vector<T*> dc(S.size()), dn(S.size());
    for (size_t q = 0; q < S.size(); ++q) {
        dc[q] = as<T>(b.ps[S[q]]->lv[l].d0);
        dn[q] = as<T>(b.ps[S[q]]->lv[l].d1);
    }
    for (int app = 0; app < nu; ++app) {
        for (size_t q = 0; q < S.size(); ++q) {
            dc[q] = as<T>(b.ps[S[q]]->lv[l].d0);
            dn[q] = as<T>(b.ps[S[q]]->lv[l].d1);
        }
        if (app == 0 && s_zero) {
            std::vector<BVec> d;
            for (size_t q = 0; q < S.size(); ++q) {
                P& p = *b.ps[S[q]];
                Level& L = p.lv[l];
                BVec v = bv0();
                v.g = L.g;
                v.x = L.b;       // b
                v.y = L.r;       // r = b
                v.y2 = dc[q];    // d = b / theta
                v.x2 = L.s;      // s = 0
                v.cheb = L.cheb;
                v.ep = eps_params(p, l, o.eps_mode_pc);
                v.slot = L.eps_d;
                v.partials = p.red->partial;
                v.counter = &p.red->counter[0];
                d.push_back(v);
            }
            JFNK_TRY(bvec<T>(b, A, BOp::CHEB_START, d, sizes));
        } else {
            std::vector<StencilArgs<T>> args;
            for (size_t q = 0; q < S.size(); ++q) {
                P& p = *b.ps[S[q]];
                Level& L = p.lv[l];
                StencilArgs<T> a = base_args<T>(p, l);
                a.u = as<T>(L.x);
                a.v = as<T>(L.s);
                a.eps = L.eps_s;
                a.Au = as<T>(L.Ax);
                a.rhs = as<T>(L.b);
                a.out = as<T>(L.r);
                a.out2 = dc[q];
                a.cheb = L.cheb;
                a.cheb_step = 0;
                a.red = RedOut::EPS;
                a.red_eps = L.eps_d;
                a.epsp = eps_params(p, l, o.eps_mode_pc);
                args.push_back(a);
                p.nF[l]++;
            }
            JFNK_TRY(bstencil<T>(b, A, Mode::CHEB0, S, l, args));
        }
        for (int i = 0; i <= k - 2; ++i) {
            std::vector<StencilArgs<T>> args;
            for (size_t q = 0; q < S.size(); ++q) {
                P& p = *b.ps[S[q]];
                Level& L = p.lv[l];
                StencilArgs<T> a = base_args<T>(p, l);
                a.u = as<T>(L.x);
                a.v = dc[q];
                a.eps = L.eps_d;
                a.Au = as<T>(L.Ax);
                a.r = as<T>(L.r);
                a.s = as<T>(L.s);
                a.dnew = dn[q];
                a.cheb = L.cheb;
                a.cheb_step = i;
                a.red = RedOut::EPS;
                a.epsp = eps_params(p, l, o.eps_mode_pc);
                a.red_eps = (i < k - 2) ? L.eps_d : L.eps_s;
                args.push_back(a);
                p.nF[l]++;
                std::swap(dc[q], dn[q]);
            }
            JFNK_TRY(bstencil<T>(b, A, i < k - 2 ? Mode::CHEB : Mode::CHEBLAST, S, l, args));
        }
    }
    return JFNK_OK;
}

// One batched V-cycle (Alg. 1) of instances `act`: lv[L_i].b -> lv[L_i].s
template <typename T>
static jfnk_status bvcycle(BCtx& b, Arena& A, const std::vector<int>& act) {
    const jfnk_options& o = *b.o;
    int cmax = 0;
    for (int i : act) cmax = std::max(cmax, b.ps[i]->L);
    auto subset = [&](int c) {
        std::vector<int> S;
        for (int i : act)
            if (b.ps[i]->L >= c) S.push_back(i);
        return S;
    };
    for (int c = cmax; c >= 1; --c) {
        const std::vector<int> S = subset(c);
        if (o.nu_pre == 0) {
            std::vector<BScal> d;
            for (int i : S) {
                BScal v;
                memset(&v, 0, sizeof(v));
                v.slot = b.ps[i]->lv[c].eps_s;
                v.a = 0.0;
                d.push_back(v);
            }
            JFNK_TRY(bscalar(b, A, BScalar::SET_EPS, d));
        }
        JFNK_TRY(bsmooth<T>(b, A, c, S, o.nu_pre, true));
        std::vector<StencilArgs<T>> args;
        std::vector<BVec> rd;
        std::vector<long long> csz;
        for (int i : S) {
            P& p = *b.ps[i];
            Level& L = p.lv[c];
            Level& C = p.lv[c - 1];
            StencilArgs<T> a = base_args<T>(p, c);
            a.u = as<T>(L.x);
            a.v = as<T>(L.s);
            a.eps = L.eps_s;
            a.Au = as<T>(L.Ax);
            a.rhs = as<T>(L.b);
            a.out = as<T>(L.t);
            args.push_back(a);
            p.nF[c]++;
            BVec v = bv0();
            v.g = L.g;
            v.gc = C.g;
            v.x = L.t;
            v.y = C.b;
            v.a = 1.0;
            v.what = 0;
            rd.push_back(v);
            csz.push_back(C.g.size);
        }
        JFNK_TRY(bstencil<T>(b, A, Mode::BMJ, S, c, args));
        JFNK_TRY(bvec<T>(b, A, BOp::RESTRICT, rd, csz));
    }
    {
        std::vector<CoarseArgs<T>> ca;
        for (int i : act) {
            P& p = *b.ps[i];
            Level& L = p.lv[0];
            CoarseArgs<T> a;
            memset(&a, 0, sizeof(a));
            a.g = L.g;
            a.x = as<T>(L.x);
            a.Ax = as<T>(L.Ax);
            a.b = as<T>(L.b);
            a.s = as<T>(L.s);
            a.lh = (T)(p.desc.lambda * L.h * L.h / 16.0);
            a.node_scale = (T)1.0;
            a.eps_mode = o.eps_mode_pc;
            a.n_unknowns = (double)L.g.interior();
            a.xstat = (o.eps_mode_pc == JFNK_EPS_PAPER) ? L.xstat_paper : L.xstat_fp32;
            a.tol = o.coarse_tol;
            a.tol_abs = o.coarse_tol_mode;
            a.maxit = p.coarse_maxit;
            a.V = as<T>(p.coarseV);
            a.H = p.coarseH;
            a.iters = p.coarse_iters;
            ca.push_back(a);
        }
        jfnk_status err = JFNK_OK;
        const CoarseArgs<T>* dca = stage(b, A, ca, err);
        if (err != JFNK_OK) return err;
        if (!b.dry) JFNK_TRY(launch_coarse_batched<T>(ca[0], dca, (int)ca.size(), b.st));
    }
    for (int c = 1; c <= cmax; ++c) {
        const std::vector<int> S = subset(c);
        std::vector<BVec> pd, nd;
        std::vector<long long> fsz;
        for (int i : S) {
            P& p = *b.ps[i];
            Level& L = p.lv[c];
            Level& C = p.lv[c - 1];
            BVec v = bv0();
            v.g = L.g;
            v.gc = C.g;
            v.x = C.s;
            v.y = L.s;
            pd.push_back(v);
            BVec w = bv0();
            w.g = L.g;
            w.x = L.s;
            w.what = 1;
            w.slot = L.eps_s;
            w.ep = eps_params(p, c, o.eps_mode_pc);
            w.partials = p.red->partial;
            w.counter = &p.red->counter[0];
            nd.push_back(w);
            fsz.push_back(L.g.size);
        }
        JFNK_TRY(bvec<T>(b, A, BOp::PROLONG_ADD, pd, fsz));
        JFNK_TRY(bvec<T>(b, A, BOp::STAT, nd, fsz));
        JFNK_TRY(bsmooth<T>(b, A, c, S, o.nu_post, false));
    }
    return JFNK_OK;
}

// Build (dry pass + upload) or reuse the V-cycle program for `act`, then run it.
template <typename T>
static jfnk_status bvcycle_run(BCtx& b, const std::vector<int>& act) {
    Arena& A = b.prog;
    std::vector<long long> nF0(b.B * JFNK_MAX_LEVELS);
    if (act != b.prog_set) {
        if (b.graph) {
            cudaGraphExecDestroy(b.graph);
            b.graph = nullptr;
        }
        A.reset();
        for (int i = 0; i < b.B; ++i) memcpy(&nF0[i * JFNK_MAX_LEVELS], b.ps[i]->nF, sizeof(long long) * JFNK_MAX_LEVELS);
        b.dry = true;
        jfnk_status s = bvcycle<T>(b, A, act);
        b.dry = false;
        for (int i = 0; i < b.B; ++i) memcpy(b.ps[i]->nF, &nF0[i * JFNK_MAX_LEVELS], sizeof(long long) * JFNK_MAX_LEVELS);
        JFNK_TRY(s);
        JFNK_CUDA_TRY(cudaMemcpyAsync(A.dev, A.host.data(), A.off, cudaMemcpyHostToDevice, b.st));
        JFNK_CUDA_TRY(cudaStreamSynchronize(b.st));
        b.prog_set = act;
    }
    A.off = 0;
    A.replay = true;
    jfnk_status s = JFNK_OK;
    if (b.o->use_graph) {
        if (!b.graph) {
            P& lp = *b.lead;
            if (!lp.cap_stream) JFNK_CUDA_TRY(cudaStreamCreateWithFlags(&lp.cap_stream, cudaStreamNonBlocking));
            cudaStream_t keep = b.st;
            b.st = lp.cap_stream;
            for (int i = 0; i < b.B; ++i) memcpy(&nF0[i * JFNK_MAX_LEVELS], b.ps[i]->nF, sizeof(long long) * JFNK_MAX_LEVELS);
            JFNK_CUDA_TRY(cudaStreamBeginCapture(lp.cap_stream, cudaStreamCaptureModeThreadLocal));
            s = bvcycle<T>(b, A, act);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(lp.cap_stream, &g);
            b.st = keep;
            for (int i = 0; i < b.B; ++i) memcpy(b.ps[i]->nF, &nF0[i * JFNK_MAX_LEVELS], sizeof(long long) * JFNK_MAX_LEVELS);
            if (s != JFNK_OK) {
                if (e == cudaSuccess && g) cudaGraphDestroy(g);
                A.replay = false;
                return s;
            }
            JFNK_CUDA_TRY(e);
            cudaError_t ei = cudaGraphInstantiate(&b.graph, g, 0);
            cudaGraphDestroy(g);
            JFNK_CUDA_TRY(ei);
            A.off = 0;
        }
        JFNK_CUDA_TRY(cudaGraphLaunch(b.graph, b.st));
        // count the evaluations of the replayed cycle (dry bookkeeping pass)
        b.dry = true;
        A.off = 0;
        s = bvcycle<T>(b, A, act);
        b.dry = false;
    } else {
        s = bvcycle<T>(b, A, act);
    }
    A.replay = false;
    return s;
}

// ---------------------------------------------------------------------------
// per-instance helpers for the dynamic (non-program) operations
static std::vector<long long> sizes_of(const BCtx& b, const std::vector<int>& S, int lvl /* -1: finest */) {
    std::vector<long long> z;
    for (int i : S) z.push_back(b.ps[i]->lv[lvl < 0 ? b.ps[i]->L : lvl].g.size);
    return z;
}

static jfnk_status read_res(BCtx& b, std::vector<double>& host) {
    host.resize((size_t)b.B * kResStride);
    JFNK_CUDA_TRY(cudaMemcpyAsync(host.data(), b.res, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, b.st));
    JFNK_CUDA_TRY(cudaStreamSynchronize(b.st));
    return JFNK_OK;
}

// out[i] = ||x_i|| (what 1) or sum |x_i| (what 0) over interior nodes; slot (optional) = FD step
static jfnk_status bstat(BCtx& b, const std::vector<int>& S, int lvl, int what, const std::vector<const void*>& x,
                         std::vector<double*> out, std::vector<EpsSlot*> slot, std::vector<EpsParams> ep, bool f64) {
    std::vector<BVec> d;
    for (size_t q = 0; q < S.size(); ++q) {
        P& p = *b.ps[S[q]];
        BVec v = bv0();
        v.g = p.lv[lvl < 0 ? p.L : lvl].g;
        v.x = x[q];
        v.what = what;
        v.out = out[q];
        v.slot = slot.empty() ? nullptr : slot[q];
        if (!ep.empty()) v.ep = ep[q];
        v.partials = p.red->partial;
        v.counter = &p.red->counter[0];
        d.push_back(v);
    }
    if (f64) return bvec<double>(b, b.dyn, BOp::STAT, d, sizes_of(b, S, lvl));
    return bvec<float>(b, b.dyn, BOp::STAT, d, sizes_of(b, S, lvl));
}

static EpsParams outer_eps(P& p) {
    EpsParams e;
    e.mode = JFNK_EPS_PAPER;
    e.n_unknowns = (double)p.lv[p.L].g.interior();
    e.xstat = p.xstat64;
    return e;
}

// w_i = J(u_i) v_i in FP64 (paper eps), instances S
static jfnk_status bjv64(BCtx& b, const std::vector<int>& S, const std::vector<const double*>& v,
                         const std::vector<double*>& w) {
    std::vector<const void*> xv;
    std::vector<double*> outs;
    std::vector<EpsSlot*> slots;
    std::vector<EpsParams> eps;
    for (size_t q = 0; q < S.size(); ++q) {
        P& p = *b.ps[S[q]];
        xv.push_back(v[q]);
        outs.push_back(nullptr);
        slots.push_back(p.eps64);
        eps.push_back(outer_eps(p));
    }
    JFNK_TRY(bstat(b, S, -1, 1, xv, outs, slots, eps, true));
    std::vector<StencilArgs<double>> args;
    for (size_t q = 0; q < S.size(); ++q) {
        P& p = *b.ps[S[q]];
        StencilArgs<double> a = base_args<double>(p, p.L);
        a.u = b.u[S[q]];
        a.v = v[q];
        a.eps = p.eps64;
        a.Au = p.Au64;
        a.out = w[q];
        args.push_back(a);
        p.nF[p.L]++;
    }
    // finest grids of different sizes: the 2D tiles carry each instance's grid
    std::vector<Grid> gs;
    for (int i : S) gs.push_back(b.ps[i]->lv[b.ps[i]->L].g);
    jfnk_status err = JFNK_OK;
    const TileCfg& tc = b.tile[1];
    const std::vector<BTile> tiles = tiles_for(gs, tc.bx, tc.target);
    const StencilArgs<double>* da = stage(b, b.dyn, args, err);
    const BTile* dt = stage(b, b.dyn, tiles, err);
    JFNK_TRY(err);
    return launch_stencil2d_batched<double>(Mode::JV, da, dt, (int)tiles.size(), tc.bx, b.st, tc.grid);
}

// F_i = F(x_i), A_i = A(x_i) (FP64, finest) and ||F_i|| into res slot 0
static jfnk_status bresidual64(BCtx& b, const std::vector<int>& S, const std::vector<const double*>& x,
                               const std::vector<double*>& F, const std::vector<double*>& Au) {
    std::vector<StencilArgs<double>> args;
    std::vector<Grid> gs;
    for (size_t q = 0; q < S.size(); ++q) {
        P& p = *b.ps[S[q]];
        StencilArgs<double> a = base_args<double>(p, p.L);
        a.u = x[q];
        a.out = F[q];
        a.out2 = Au[q];
        args.push_back(a);
        gs.push_back(p.lv[p.L].g);
        p.nF[p.L]++;
        p.nFplain[p.L]++;
    }
    jfnk_status err = JFNK_OK;
    const TileCfg& tc = b.tile[1];
    const std::vector<BTile> tiles = tiles_for(gs, tc.bx, tc.target);
    const StencilArgs<double>* da = stage(b, b.dyn, args, err);
    const BTile* dt = stage(b, b.dyn, tiles, err);
    JFNK_TRY(err);
    JFNK_TRY(launch_stencil2d_batched<double>(Mode::F, da, dt, (int)tiles.size(), tc.bx, b.st, tc.grid));
    std::vector<const void*> xv(F.begin(), F.end());
    std::vector<double*> outs;
    for (int i : S) outs.push_back(b.res + (size_t)i * kResStride);
    return bstat(b, S, -1, 1, xv, outs, {}, {}, true);
}

// y_i = a_i x_i + c_i y_i (FP64, finest)
static jfnk_status baxpby(BCtx& b, const std::vector<int>& S, const std::vector<double*>& y,
                          const std::vector<const double*>& x, const std::vector<double>& a,
                          const std::vector<double>& c, const std::vector<const double*>& x2 = {}) {
    std::vector<BVec> d;
    for (size_t q = 0; q < S.size(); ++q) {
        P& p = *b.ps[S[q]];
        BVec v = bv0();
        v.g = p.lv[p.L].g;
        v.y = y[q];
        v.x = x[q];
        v.a = a[q];
        v.b = c[q];
        if (!x2.empty()) v.x2 = x2[q];
        d.push_back(v);
    }
    return bvec<double>(b, b.dyn, x2.empty() ? BOp::AXPBY_D : BOp::ADDSC_D, d, sizes_of(b, S, -1));
}

// x_l, A(x_l), statistics and lambda_l (power method) of instances S (Sec. 2)
template <typename T>
static jfnk_status bsetup(BCtx& b, const std::vector<int>& S, int newton_step) {
    const jfnk_options& o = *b.o;
    Arena& A = b.dyn;
    int cmax = 0;
    for (int i : S) cmax = std::max(cmax, b.ps[i]->L);
    auto subset = [&](int c) {
        std::vector<int> R;
        for (int i : S)
            if (b.ps[i]->L >= c) R.push_back(i);
        return R;
    };
    {
        std::vector<BVec> d;
        for (int i : S) {
            P& p = *b.ps[i];
            BVec v = bv0();
            v.g = p.lv[p.L].g;
            v.x = b.u[i];
            v.y = p.lv[p.L].x;
            d.push_back(v);
        }
        JFNK_TRY(bvec<T>(b, A, BOp::CAST_D2T, d, sizes_of(b, S, -1)));
    }
    for (int c = cmax; c >= 1; --c) {
        const std::vector<int> R = subset(c);
        std::vector<BVec> d;
        std::vector<long long> z;
        for (int i : R) {
            P& p = *b.ps[i];
            BVec v = bv0();
            v.g = p.lv[c].g;
            v.gc = p.lv[c - 1].g;
            v.x = p.lv[c].x;
            v.y = p.lv[c - 1].x;
            v.a = 0.25;  // 2^-d
            v.what = 1;  // projection: boundary injection
            d.push_back(v);
            z.push_back(p.lv[c - 1].g.size);
        }
        JFNK_TRY(bvec<T>(b, A, BOp::RESTRICT, d, z));
    }
    for (int c = 0; c <= cmax; ++c) {
        const std::vector<int> R = subset(c);
        std::vector<StencilArgs<T>> args;
        std::vector<const void*> xv;
        std::vector<double*> o1, o2;
        for (int i : R) {
            P& p = *b.ps[i];
            StencilArgs<T> a = base_args<T>(p, c);
            a.u = as<T>(p.lv[c].x);
            a.out = as<T>(p.lv[c].Ax);
            args.push_back(a);
            p.nF[c]++;
            p.nFplain[c]++;
            xv.push_back(p.lv[c].x);
            o1.push_back(p.lv[c].xstat_paper);
            o2.push_back(p.lv[c].xstat_fp32);
        }
        JFNK_TRY(bstencil<T>(b, A, Mode::F, R, c, args));
        JFNK_TRY(bstat(b, R, c, 0, xv, o1, {}, {}, sizeof(T) == 8));
        JFNK_TRY(bstat(b, R, c, 1, xv, o2, {}, {}, sizeof(T) == 8));
    }
    // Power method on every smoothed level of every instance.  Levels and
    // instances are independent: each round issues one iteration for every
    // (level, instance) still running, and with the stopping rule on
    // (power_tol > 0) the host reads all their estimates with one
    // synchronisation per round and drops each pair once its estimate settles.
    std::vector<std::vector<int>> Rl(cmax + 1);
    for (int c = 1; c <= cmax; ++c) {
        const std::vector<int> R = subset(c);
        Rl[c] = R;
        if (R.empty()) continue;
        const std::vector<long long> z = sizes_of(b, R, c);
        std::vector<const void*> pv;
        std::vector<EpsParams> ep;
        std::vector<EpsSlot*> slots;
        std::vector<double*> n0;
        std::vector<BVec> start, sc;
        for (int i : R) {
            Level& L = b.ps[i]->lv[c];
            pv.push_back(L.pv);
            ep.push_back(eps_params(*b.ps[i], c, o.eps_mode_pc));
            slots.push_back(L.eps_aux);
            n0.push_back(L.nrm0);
            BVec v = bv0();
            v.g = L.g;
            v.y = L.pv;
            v.key = o.seed + (uint64_t)c * 0xD1B54A32D192ED03ULL;
            start.push_back(v);
            BVec w = bv0();
            w.g = L.g;
            w.x = w.y = L.pv;
            w.dsc = L.nrm0;
            sc.push_back(w);
        }
        if (newton_step == 0 || !b.ps[R[0]]->lv[c].pv_valid) JFNK_TRY(bvec<T>(b, A, BOp::SPLITMIX, start, z));
        // v <- v / ||v||
        JFNK_TRY(bstat(b, R, c, 1, pv, n0, slots, ep, sizeof(T) == 8));
        JFNK_TRY(bvec<T>(b, A, BOp::SCALE_INV_T, sc, z));
    }
    // one iteration on level c for instances Ra: w = J v (FD), lambda = ||w|| / ||v||,
    // v <- w / ||w||
    auto iterate = [&](int c, const std::vector<int>& Ra) -> jfnk_status {
        std::vector<const void*> pv;
        std::vector<double*> n0;
        std::vector<EpsSlot*> slots;
        std::vector<EpsParams> ep;
        std::vector<BVec> sc;
        std::vector<long long> z;
        std::vector<StencilArgs<T>> args;
        std::vector<BScal> rat;
        for (int i : Ra) {
            P& p = *b.ps[i];
            Level& L = p.lv[c];
            pv.push_back(L.pv);
            n0.push_back(L.nrm0);
            slots.push_back(L.eps_aux);
            ep.push_back(eps_params(p, c, o.eps_mode_pc));
            BVec v = bv0();
            v.g = L.g;
            v.x = v.y = L.pw;
            v.dsc = L.nrm1;
            sc.push_back(v);
            z.push_back(L.g.size);
            StencilArgs<T> a = base_args<T>(p, c);
            a.u = as<T>(L.x);
            a.v = as<T>(L.pv);
            a.eps = L.eps_aux;
            a.Au = as<T>(L.Ax);
            a.out = as<T>(L.pw);
            a.red = RedOut::NORM;
            a.red_norm = L.nrm1;
            args.push_back(a);
            p.nF[c]++;
            BScal r;
            memset(&r, 0, sizeof(r));
            r.out = L.lam;
            r.x = L.nrm1;
            r.x2 = L.nrm0;
            rat.push_back(r);
        }
        JFNK_TRY(bstat(b, Ra, c, 1, pv, n0, slots, ep, sizeof(T) == 8));
        JFNK_TRY(bstencil<T>(b, A, Mode::JV, Ra, c, args));
        JFNK_TRY(bscalar(b, A, BScalar::RATIO, rat));
        JFNK_TRY(bvec<T>(b, A, BOp::SCALE_INV_T, sc, z));
        for (int i : Ra) std::swap(b.ps[i]->lv[c].pv, b.ps[i]->lv[c].pw);
        return JFNK_OK;
    };
    std::vector<std::vector<double>> lam_prev(cmax + 1, std::vector<double>(b.ps.size(), 0.0));
    std::vector<std::vector<double>> lam_now = lam_prev;
    for (int it = 0; it < o.power_iters; ++it) {
        bool any = false;
        for (int c = 1; c <= cmax; ++c) {
            if (Rl[c].empty()) continue;
            any = true;
            JFNK_TRY(iterate(c, Rl[c]));
        }
        if (!any) break;
        if (o.power_tol > 0.0) {
            for (int c = 1; c <= cmax; ++c)
                for (int i : Rl[c])
                    JFNK_CUDA_TRY(cudaMemcpyAsync(&lam_now[c][i], b.ps[i]->lv[c].lam, sizeof(double),
                                                  cudaMemcpyDeviceToHost, b.st));
            JFNK_CUDA_TRY(cudaStreamSynchronize(b.st));
            for (int c = 1; c <= cmax; ++c) {
                std::vector<int> still;
                for (int i : Rl[c]) {
                    const bool done =
                        it > 0 && std::fabs(lam_now[c][i] - lam_prev[c][i]) < o.power_tol * lam_now[c][i];
                    lam_prev[c][i] = lam_now[c][i];
                    if (!done) still.push_back(i);
                }
                Rl[c].swap(still);
            }
        }
    }
    for (int c = 1; c <= cmax; ++c) {
        const std::vector<int> R = subset(c);
        std::vector<BScal> ct;
        for (int i : R) {
            P& p = *b.ps[i];
            p.lv[c].pv_valid = true;
            BScal t;
            memset(&t, 0, sizeof(t));
            t.x = p.lv[c].lam;
            t.a = o.cheb_lo;
            t.b = o.cheb_hi;
            t.m = o.cheb_degree;
            t.cheb = p.lv[c].cheb;
            t.status = p.status;
            ct.push_back(t);
        }
        JFNK_TRY(bscalar(b, A, BScalar::CHEB_TABLE, ct));
    }
    return JFNK_OK;
}

// Lock-step FGMRES(m) for instances S: J(u_i) delta_i = rhs64_i to eta_i ||rhs_i||.
template <typename T>
static jfnk_status bfgmres(BCtx& b, const std::vector<int>& S, const std::vector<double>& eta, std::vector<int>& its,
                           std::vector<ArnoldiSlope>& slope) {
    const jfnk_options& o = *b.o;
    const int m = o.restart;
    std::vector<double> hr;
    // delta = 0, beta0 = ||rhs||, tmp = rhs
    {
        std::vector<double*> y;
        std::vector<const double*> x;
        for (int i : S) {
            y.push_back(b.ps[i]->delta);
            x.push_back(b.ps[i]->delta);
        }
        JFNK_TRY(baxpby(b, S, y, x, std::vector<double>(S.size(), 0.0), std::vector<double>(S.size(), 0.0)));
        std::vector<double*> t;
        std::vector<const double*> r;
        for (int i : S) {
            t.push_back(b.ps[i]->tmp64);
            r.push_back(b.ps[i]->rhs64);
        }
        JFNK_TRY(baxpby(b, S, t, r, std::vector<double>(S.size(), 1.0), std::vector<double>(S.size(), 0.0)));
        std::vector<const void*> xv(r.begin(), r.end());
        std::vector<double*> outs;
        for (int i : S) outs.push_back(b.res + (size_t)i * kResStride);
        JFNK_TRY(bstat(b, S, -1, 1, xv, outs, {}, {}, true));
    }
    JFNK_TRY(read_res(b, hr));
    std::vector<double> target(b.B, 0.0), beta(b.B, 0.0);
    std::vector<int> act;
    for (size_t q = 0; q < S.size(); ++q) {
        const int i = S[q];
        its[i] = 0;
        beta[i] = hr[(size_t)i * kResStride];
        if (!std::isfinite(beta[i])) {
            set_error("non-finite right-hand side in batched FGMRES (instance %d)", i);
            return JFNK_ERR_NONFINITE;
        }
        target[i] = eta[q] * beta[i];
        if (beta[i] > 0.0 && beta[i] > target[i]) act.push_back(i);
    }
    std::vector<std::vector<double>> H(b.B), Hraw(b.B), g(b.B), cs(b.B), sn(b.B);
    std::vector<int> k(b.B, 0);
    for (int i : S) slope[i] = ArnoldiSlope();
    while (!act.empty()) {
        // V_0 = tmp / beta (beta already in res slot 0)
        {
            std::vector<BVec> d;
            for (int i : act) {
                P& p = *b.ps[i];
                BVec v = bv0();
                v.g = p.lv[p.L].g;
                v.x = p.tmp64;
                v.y = p.V64;
                v.dsc = b.res + (size_t)i * kResStride;
                d.push_back(v);
                H[i].assign((size_t)(m + 1) * m, 0.0);
                Hraw[i].assign((size_t)(m + 1) * m, 0.0);
                slope[i].cycles++;
                slope[i].beta = beta[i];
                g[i].assign(m + 1, 0.0);
                cs[i].assign(m, 0.0);
                sn[i].assign(m, 0.0);
                g[i][0] = beta[i];
                k[i] = 0;
            }
            JFNK_TRY(bvec<double>(b, b.dyn, BOp::SCALE_INV_T, d, sizes_of(b, act, -1)));
        }
        std::vector<int> run = act;
        std::vector<char> conv(b.B, 0);
        for (int j = 0; j < m && !run.empty(); ++j) {
            // z_j = MG(v_j)
            std::vector<BVec> cd, zd, zd64;
            for (int i : run) {
                P& p = *b.ps[i];
                const long long N = p.lv[p.L].g.size;
                BVec v = bv0();
                v.g = p.lv[p.L].g;
                v.x = p.V64 + (size_t)j * N;
                v.y = p.lv[p.L].b;
                cd.push_back(v);
                BVec z = bv0();
                z.g = p.lv[p.L].g;
                z.x = p.lv[p.L].s;
                z.y = as<T>(p.Z) + (size_t)j * N;
                zd.push_back(z);
                BVec z2 = bv0();
                z2.g = p.lv[p.L].g;
                z2.x = as<T>(p.Z) + (size_t)j * N;
                z2.y = p.z64;
                zd64.push_back(z2);
            }
            JFNK_TRY(bvec<T>(b, b.dyn, BOp::CAST_D2T, cd, sizes_of(b, run, -1)));
            JFNK_TRY(bvcycle_run<T>(b, run));
            JFNK_TRY(bvec<T>(b, b.dyn, BOp::COPY_T, zd, sizes_of(b, run, -1)));
            std::vector<const double*> zv;
            std::vector<double*> wv;
            if (sizeof(T) == 8) {
                for (size_t q = 0; q < run.size(); ++q) zv.push_back((const double*)zd[q].y);
            } else {
                JFNK_TRY(bvec<T>(b, b.dyn, BOp::CAST_T2D, zd64, sizes_of(b, run, -1)));
                for (int i : run) zv.push_back(b.ps[i]->z64);
            }
            for (int i : run) wv.push_back(b.ps[i]->w64);
            JFNK_TRY(bjv64(b, run, zv, wv));
            // classical Gram-Schmidt twice, then ||w||
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<BVec> dd;
                for (int i : run) {
                    P& p = *b.ps[i];
                    BVec v = bv0();
                    v.g = p.lv[p.L].g;
                    v.x = p.w64;
                    v.y = p.w64;
                    v.x2 = p.V64;
                    v.ld = p.lv[p.L].g.size;
                    v.m = j + 1;
                    v.out = b.res + (size_t)i * kResStride + 1 + pass * (m + 2);
                    v.partials = p.dot_partials;
                    v.counter = &p.counters[2];
                    dd.push_back(v);
                }
                JFNK_TRY(bvec<double>(b, b.dyn, BOp::MDOT, dd, sizes_of(b, run, -1)));
                JFNK_TRY(bvec<double>(b, b.dyn, BOp::MAXPY_SUB, dd, sizes_of(b, run, -1)));
            }
            {
                std::vector<const void*> xv;
                std::vector<double*> outs;
                for (int i : run) {
                    xv.push_back(b.ps[i]->w64);
                    outs.push_back(b.res + (size_t)i * kResStride + 2 * (m + 2) + 1);
                }
                JFNK_TRY(bstat(b, run, -1, 1, xv, outs, {}, {}, true));
            }
            JFNK_TRY(read_res(b, hr));
            std::vector<int> next;
            for (int i : run) {
                const double* rr = &hr[(size_t)i * kResStride];
                double* col = &H[i][(size_t)j * (m + 1)];
                for (int q = 0; q <= j; ++q) col[q] = rr[1 + q] + rr[1 + (m + 2) + q];
                const double hn = rr[2 * (m + 2) + 1];
                col[j + 1] = hn;
                for (int q = 0; q <= j + 1; ++q) Hraw[i][(size_t)j * (m + 1) + q] = col[q];
                if (!std::isfinite(hn)) {
                    set_error("non-finite Arnoldi entry in batched FGMRES (instance %d)", i);
                    return JFNK_ERR_NONFINITE;
                }
                for (int q = 0; q < j; ++q) {
                    const double t = cs[i][q] * col[q] + sn[i][q] * col[q + 1];
                    col[q + 1] = -sn[i][q] * col[q] + cs[i][q] * col[q + 1];
                    col[q] = t;
                }
                givens(col[j], col[j + 1], cs[i][j], sn[i][j]);
                col[j] = cs[i][j] * col[j] + sn[i][j] * col[j + 1];
                col[j + 1] = 0.0;
                g[i][j + 1] = -sn[i][j] * g[i][j];
                g[i][j] = cs[i][j] * g[i][j];
                const double res = std::fabs(g[i][j + 1]);
                k[i] = j + 1;
                its[i]++;
                if (res <= target[i] || hn == 0.0) conv[i] = 1;
                if (conv[i] || its[i] >= o.max_linear) continue;
                next.push_back(i);
            }
            if (!next.empty() && j + 1 < m) {
                std::vector<BVec> d;
                for (int i : next) {
                    P& p = *b.ps[i];
                    BVec v = bv0();
                    v.g = p.lv[p.L].g;
                    v.x = p.w64;
                    v.y = p.V64 + (size_t)(j + 1) * p.lv[p.L].g.size;
                    v.dsc = b.res + (size_t)i * kResStride + 2 * (m + 2) + 1;
                    d.push_back(v);
                }
                JFNK_TRY(bvec<double>(b, b.dyn, BOp::SCALE_INV_T, d, sizes_of(b, next, -1)));
            }
            run = next;
        }
        // y = H^-1 g ; delta += Z y (coefficients staged in res slots 1..k)
        std::vector<double> yall((size_t)b.B * kResStride, 0.0);
        for (int i : act) {
            std::vector<double> y(k[i]);
            for (int q = k[i] - 1; q >= 0; --q) {
                const double hqq = H[i][(size_t)q * (m + 1) + q];
                if (hqq == 0.0) {
                    set_error("FGMRES breakdown in instance %d: singular Hessenberg matrix at column %d", i, q);
                    return JFNK_ERR_BREAKDOWN;
                }
                double t = g[i][q];
                for (int r = q + 1; r < k[i]; ++r) t -= H[i][(size_t)r * (m + 1) + q] * y[r];
                y[q] = t / hqq;
            }
            for (int q = 0; q < k[i]; ++q) yall[(size_t)i * kResStride + 1 + q] = y[q];
            double hy0 = 0.0;
            for (int q = 0; q < k[i]; ++q) hy0 += Hraw[i][(size_t)q * (m + 1)] * y[q];
            slope[i].Hy0 = hy0;
        }
        JFNK_CUDA_TRY(cudaMemcpyAsync(b.res, yall.data(), sizeof(double) * yall.size(), cudaMemcpyHostToDevice, b.st));
        {
            std::vector<BVec> d;
            for (int i : act) {
                P& p = *b.ps[i];
                BVec v = bv0();
                v.g = p.lv[p.L].g;
                v.y = p.delta;
                v.x = p.Z;
                v.ld = p.lv[p.L].g.size;
                v.m = k[i];
                v.dsc = b.res + (size_t)i * kResStride + 1;
                d.push_back(v);
            }
            JFNK_TRY(bvec<T>(b, b.dyn, BOp::COMBINE_T, d, sizes_of(b, act, -1)));
        }
        // instances that neither converged nor ran out restart from r = rhs - J delta
        std::vector<int> rest;
        for (int i : act)
            if (!conv[i] && its[i] < o.max_linear) rest.push_back(i);
        if (rest.empty()) break;
        std::vector<const double*> dv;
        std::vector<double*> wv;
        for (int i : rest) {
            dv.push_back(b.ps[i]->delta);
            wv.push_back(b.ps[i]->w64);
        }
        JFNK_TRY(bjv64(b, rest, dv, wv));
        std::vector<double*> t;
        std::vector<const double*> r, w2;
        for (int i : rest) {
            t.push_back(b.ps[i]->tmp64);
            r.push_back(b.ps[i]->rhs64);
            w2.push_back(b.ps[i]->w64);
        }
        JFNK_TRY(baxpby(b, rest, t, r, std::vector<double>(rest.size(), -1.0), std::vector<double>(rest.size(), 0.0),
                        w2));
        std::vector<const void*> xv(t.begin(), t.end());
        std::vector<double*> outs;
        for (int i : rest) outs.push_back(b.res + (size_t)i * kResStride);
        JFNK_TRY(bstat(b, rest, -1, 1, xv, outs, {}, {}, true));
        JFNK_TRY(read_res(b, hr));
        act.clear();
        for (int i : rest) {
            beta[i] = hr[(size_t)i * kResStride];
            if (beta[i] > target[i]) act.push_back(i);
        }
    }
    return JFNK_OK;
}

// ---------------------------------------------------------------------------
// Tile autotuner: the first batched solve of a given mix of grid sizes times
// the residual kernel of the finest grids for a few (threads per CTA, target
// CTA count, persistent grid) candidates with CUDA events and keeps the
// fastest, per precision.  Results are cached in the process and, when the
// environment variable JFNK_TUNE_CACHE names a file, in that file (one line
// per key: "key bx target grid ms").
static std::map<std::string, TileCfg>& tile_cache() {
    static std::map<std::string, TileCfg> m;
    static bool loaded = false;
    if (!loaded) {
        loaded = true;
        const char* path = getenv("JFNK_TUNE_CACHE");
        if (path) {
            FILE* f = fopen(path, "r");
            if (f) {
                char key[512];
                TileCfg c;
                double ms;
                while (fscanf(f, "%511s %d %d %d %lf", key, &c.bx, &c.target, &c.grid, &ms) == 5) m[key] = c;
                fclose(f);
            }
        }
    }
    return m;
}

static void tile_cache_store(const std::string& key, const TileCfg& c, double ms) {
    tile_cache()[key] = c;
    const char* path = getenv("JFNK_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), c.bx, c.target, c.grid, ms);
    fclose(f);
}

template <typename T>
static jfnk_status tune_tiles(BCtx& b) {
    const int ti = sizeof(T) == 8 ? 1 : 0;
    std::vector<int> ns;
    for (P* p : b.ps) ns.push_back(p->lv[p->L].g.n);
    std::sort(ns.begin(), ns.end());
    std::string key = std::string("bratu2d_") + (ti ? "f64" : "f32");
    for (size_t k = 0; k < ns.size();) {
        size_t e = k;
        while (e < ns.size() && ns[e] == ns[k]) ++e;
        key += "_" + std::to_string(ns[k]) + "x" + std::to_string(e - k);
        k = e;
    }
    auto it = tile_cache().find(key);
    if (it != tile_cache().end()) {
        b.tile[ti] = it->second;
        return JFNK_OK;
    }
    std::vector<int> all(b.B);
    std::vector<Grid> gs;
    std::vector<StencilArgs<T>> args;
    for (int i = 0; i < b.B; ++i) {
        all[i] = i;
        P& p = *b.ps[i];
        gs.push_back(p.lv[p.L].g);
        StencilArgs<T> a = base_args<T>(p, p.L);
        if (ti) {
            a.u = (const T*)b.u[i];
            a.out = (T*)p.Ftrial;
        } else {
            a.u = as<T>(p.lv[p.L].x);
            a.out = as<T>(p.lv[p.L].t);
        }
        args.push_back(a);
    }
    int dev = 0, sms = kNumSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    JFNK_CUDA_TRY(cudaEventCreate(&e0));
    JFNK_CUDA_TRY(cudaEventCreate(&e1));
    TileCfg best;
    double best_ms = -1.0;
    jfnk_status err = JFNK_OK;
    for (int bx : {128, 160, 256}) {
        for (int target : {304, 608, 1216}) {
            const std::vector<BTile> tiles = tiles_for(gs, bx, target);
            const StencilArgs<T>* da = stage(b, b.dyn, args, err);
            const BTile* dt = stage(b, b.dyn, tiles, err);
            JFNK_TRY(err);
            const int per_sm = std::max(1, 2048 / bx);
            for (int grid : {0, sms * per_sm}) {
                TileCfg c{bx, target, grid};
                JFNK_TRY(launch_stencil2d_batched<T>(Mode::F, da, dt, (int)tiles.size(), bx, b.st, grid));
                JFNK_CUDA_TRY(cudaEventRecord(e0, b.st));
                for (int r = 0; r < 3; ++r)
                    JFNK_TRY(launch_stencil2d_batched<T>(Mode::F, da, dt, (int)tiles.size(), bx, b.st, grid));
                JFNK_CUDA_TRY(cudaEventRecord(e1, b.st));
                JFNK_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                JFNK_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (best_ms < 0.0 || ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b.tile[ti] = best;
    tile_cache_store(key, best, best_ms / 3.0);
    return JFNK_OK;
}

template <typename T>
static jfnk_status bsolve(BCtx& b, jfnk_stats* stats) {
    const jfnk_options& o = *b.o;
    const int B = b.B;
    std::vector<int> all(B);
    for (int i = 0; i < B; ++i) {
        all[i] = i;
        for (int l = 0; l <= b.ps[i]->L; ++l) b.ps[i]->nF[l] = b.ps[i]->nFplain[l] = 0;
    }
    std::vector<long long> ci0(B, 0);
    for (int i = 0; i < B; ++i)
        JFNK_CUDA_TRY(cudaMemcpyAsync(&ci0[i], b.ps[i]->coarse_iters, sizeof(long long), cudaMemcpyDeviceToHost, b.st));
    JFNK_TRY(tune_tiles<double>(b));
    if (sizeof(T) == 4) JFNK_TRY(tune_tiles<T>(b));
    auto Fs = [&](const std::vector<int>& S, bool trial) {
        std::vector<double*> F, A;
        for (int i : S) {
            F.push_back(trial ? b.ps[i]->Ftrial : b.ps[i]->F64);
            A.push_back(trial ? b.ps[i]->Autrial : b.ps[i]->Au64);
        }
        return std::make_pair(F, A);
    };
    std::vector<double> hr;
    {
        auto fa = Fs(all, false);
        std::vector<const double*> x(b.u.begin(), b.u.end());
        JFNK_TRY(bresidual64(b, all, x, fa.first, fa.second));
        JFNK_TRY(read_res(b, hr));
    }
    std::vector<jfnk_stats> S(B);
    std::vector<double> F0(B), nF(B);
    for (int i = 0; i < B; ++i) {
        memset(&S[i], 0, sizeof(jfnk_stats));
        F0[i] = nF[i] = hr[(size_t)i * kResStride];
        S[i].res_hist[0] = nF[i];
    }
    auto conv = [&](int i) {
        return F0[i] == 0.0 || nF[i] <= o.rtol_newton * F0[i] || (o.atol_newton > 0.0 && nF[i] < o.atol_newton);
    };
    std::vector<char> failed(B, 0);
    for (int k = 0; k < o.max_newton; ++k) {
        std::vector<int> act;
        for (int i = 0; i < B; ++i)
            if (!conv(i) && !failed[i]) act.push_back(i);
        if (act.empty()) break;
        for (int i : act)
            if (!std::isfinite(nF[i])) {
                set_error("non-finite residual norm (instance %d, Newton step %d)", i, k);
                return JFNK_ERR_NONFINITE;
            }
        JFNK_TRY(bsetup<T>(b, act, k));
        {
            std::vector<const void*> xv;
            std::vector<double*> outs;
            for (int i : act) {
                xv.push_back(b.u[i]);
                outs.push_back(b.ps[i]->xstat64);
            }
            JFNK_TRY(bstat(b, act, -1, 0, xv, outs, {}, {}, true));
            std::vector<double*> r;
            std::vector<const double*> f;
            for (int i : act) {
                r.push_back(b.ps[i]->rhs64);
                f.push_back(b.ps[i]->F64);
            }
            JFNK_TRY(baxpby(b, act, r, f, std::vector<double>(act.size(), -1.0), std::vector<double>(act.size(), 0.0)));
        }
        std::vector<double> eta;
        for (int i : act)
            eta.push_back(o.eta_mode == 1 ? std::fmin(o.eta_max, nF[i]) : std::fmin(o.eta_max, nF[i] / F0[i]));
        std::vector<int> its(B, 0);
        std::vector<ArnoldiSlope> asl(B);
        JFNK_TRY(bfgmres<T>(b, act, eta, its, asl));
        for (int i : act) {
            JFNK_TRY(check_status(*b.ps[i], b.st));
            S[i].linear_its += its[i];
            if (k < JFNK_MAX_HIST) S[i].lin_hist[k] = its[i];
        }
        // line search: slope F . (J delta) -- from the Arnoldi relation after a
        // single FGMRES cycle, else from one more FD action -- then backtracking
        // per instance
        std::vector<double> slope(B, 0.0), alpha(B, 1.0), nT(B, 0.0), pa(B, -1.0), pf(B, 0.0);
        std::vector<int> fd;
        for (int i : act) {
            if (asl[i].cycles == 1)
                slope[i] = -asl[i].beta * asl[i].Hy0;
            else
                fd.push_back(i);
        }
        if (o.line_search && !fd.empty()) {
            std::vector<const double*> dv;
            std::vector<double*> wv;
            for (int i : fd) {
                dv.push_back(b.ps[i]->delta);
                wv.push_back(b.ps[i]->w64);
            }
            JFNK_TRY(bjv64(b, fd, dv, wv));
            std::vector<BVec> d;
            for (int i : fd) {
                P& p = *b.ps[i];
                BVec v = bv0();
                v.g = p.lv[p.L].g;
                v.x = p.F64;
                v.x2 = p.w64;
                v.ld = 0;
                v.m = 1;
                v.out = b.res + (size_t)i * kResStride + 1;
                v.partials = p.dot_partials;
                v.counter = &p.counters[2];
                d.push_back(v);
            }
            JFNK_TRY(bvec<double>(b, b.dyn, BOp::MDOT, d, sizes_of(b, fd, -1)));
            JFNK_TRY(read_res(b, hr));
            for (int i : fd) slope[i] = hr[(size_t)i * kResStride + 1];
        }
        std::vector<int> search = act;
        std::vector<char> ok(B, 0);
        std::vector<int> trials(B, 0);
        std::vector<double> tested(B, 1.0);
        for (int ls = 0; ls < (o.line_search ? o.ls_max : 1) && !search.empty(); ++ls) {
            std::vector<double*> ut;
            std::vector<const double*> uu, dd;
            std::vector<double> al;
            for (int i : search) {
                ut.push_back(b.ps[i]->utrial);
                uu.push_back(b.u[i]);
                dd.push_back(b.ps[i]->delta);
                al.push_back(alpha[i]);
            }
            JFNK_TRY(baxpby(b, search, ut, uu, al, std::vector<double>(search.size(), 0.0), dd));
            auto fa = Fs(search, true);
            std::vector<const double*> xt(ut.begin(), ut.end());
            JFNK_TRY(bresidual64(b, search, xt, fa.first, fa.second));
            JFNK_TRY(read_res(b, hr));
            std::vector<int> again;
            for (int i : search) {
                nT[i] = hr[(size_t)i * kResStride];
                trials[i]++;
                tested[i] = alpha[i];
                const double f0 = 0.5 * nF[i] * nF[i];
                const double fn = 0.5 * nT[i] * nT[i];
                if (!o.line_search || (std::isfinite(fn) && fn <= f0 + 1e-4 * alpha[i] * slope[i])) {
                    ok[i] = 1;
                    continue;
                }
                double t;
                if (!std::isfinite(fn)) {
                    // cut the step; the trial is not an interpolation point
                    alpha[i] = 0.1 * alpha[i];
                    pa[i] = -1.0;
                    again.push_back(i);
                    continue;
                } else if (pa[i] < 0.0) {
                    t = -slope[i] * alpha[i] * alpha[i] / (2.0 * (fn - f0 - slope[i] * alpha[i]));
                } else {
                    const double r1 = fn - f0 - slope[i] * alpha[i];
                    const double r2 = pf[i] - f0 - slope[i] * pa[i];
                    const double Aq = (r1 / (alpha[i] * alpha[i]) - r2 / (pa[i] * pa[i])) / (alpha[i] - pa[i]);
                    const double Bq = (-pa[i] * r1 / (alpha[i] * alpha[i]) + alpha[i] * r2 / (pa[i] * pa[i])) / (alpha[i] - pa[i]);
                    if (Aq == 0.0) {
                        t = -slope[i] / (2.0 * Bq);
                    } else {
                        const double disc = Bq * Bq - 3.0 * Aq * slope[i];
                        t = disc >= 0.0 ? (-Bq + std::sqrt(disc)) / (3.0 * Aq) : 0.5 * alpha[i];
                    }
                }
                t = std::fmin(std::fmax(t, 0.1 * alpha[i]), 0.5 * alpha[i]);
                pa[i] = alpha[i];
                pf[i] = fn;
                alpha[i] = t;
                again.push_back(i);
            }
            search = again;
        }
        // take the accepted trial of every instance; an instance whose line
        // search found no sufficient decrease keeps its iterate and stops
        // (Dennis & Schnabel, Sec. 6.3)
        std::vector<int> take;
        for (int i : act)
            if (ok[i]) take.push_back(i);
        if (!take.empty()) {
            std::vector<double*> uo;
            std::vector<const double*> ut;
            for (int i : take) {
                uo.push_back(b.u[i]);
                ut.push_back(b.ps[i]->utrial);
            }
            JFNK_TRY(baxpby(b, take, uo, ut, std::vector<double>(take.size(), 1.0),
                            std::vector<double>(take.size(), 0.0)));
        }
        for (int i : act) {
            P& p = *b.ps[i];
            S[i].newton_its = k + 1;
            if (k < JFNK_MAX_HIST) S[i].ls_hist[k] = trials[i];
            if (!ok[i]) {
                failed[i] = 1;
                S[i].status = JFNK_ERR_LINESEARCH;
                if (k + 1 < JFNK_MAX_HIST) S[i].res_hist[k + 1] = nF[i];
                if (k < JFNK_MAX_HIST) S[i].alpha_hist[k] = 0.0;
                continue;
            }
            std::swap(p.F64, p.Ftrial);
            std::swap(p.Au64, p.Autrial);
            nF[i] = nT[i];
            if (k + 1 < JFNK_MAX_HIST) S[i].res_hist[k + 1] = nF[i];
            if (k < JFNK_MAX_HIST) S[i].alpha_hist[k] = tested[i];
        }
    }
    jfnk_status result = JFNK_OK;
    for (int i = 0; i < B; ++i) {
        P& p = *b.ps[i];
        long long ci1 = 0;
        JFNK_CUDA_TRY(cudaMemcpyAsync(&ci1, p.coarse_iters, sizeof(long long), cudaMemcpyDeviceToHost, b.st));
        JFNK_CUDA_TRY(cudaStreamSynchronize(b.st));
        p.nF[0] += ci1 - ci0[i];
        double ge = 0.0;
        for (int l = 0; l <= p.L && l < JFNK_MAX_LEVELS; ++l) {
            S[i].nF[l] = p.nF[l];
            S[i].nJv[l] = p.nF[l] - p.nFplain[l];
            ge += std::pow(2.0, -2.0 * (p.L - l)) * (double)p.nF[l];
            if (l >= 1) JFNK_CUDA_TRY(cudaMemcpy(&S[i].lambda_max[l], p.lv[l].lam, sizeof(double), cudaMemcpyDeviceToHost));
        }
        S[i].ge = ge;
        S[i].converged = conv(i) ? 1 : 0;
        if (S[i].status == JFNK_OK && !S[i].converged) S[i].status = JFNK_ERR_NOT_CONVERGED;
        if (S[i].status != JFNK_OK && result == JFNK_OK) {
            result = (jfnk_status)S[i].status;
            set_error("instance %d of the batch did not converge (status %d)", i, S[i].status);
        }
        if (stats) stats[i] = S[i];
    }
    return result;
}

}  // namespace jfnk

jfnk_status jfnk_solve_batched(jfnk_problem* const* problems, int count, const jfnk_options* opts,
                               double* const* u_inout, jfnk_stats* stats, void* stream) {
    using namespace jfnk;
    if (!problems || !u_inout || count < 1) {
        set_error("jfnk_solve_batched: empty batch");
        return JFNK_ERR_INVALID_ARG;
    }
    if (opts && (opts->outer != JFNK_OUTER_FGMRES || opts->coarse_method != JFNK_COARSE_GMRES)) {
        set_error("jfnk_solve_batched: FGMRES outer and GMRES coarse solves only");
        return JFNK_ERR_NOT_IMPLEMENTED;
    }
    for (int i = 0; i < count; ++i) {
        JFNK_TRY(need_solver(problems[i], opts));
        const P& p = *problems[i];
        if (p.desc.kind != JFNK_BRATU2D || !u_inout[i]) {
            set_error("jfnk_solve_batched: instance %d is not a 2D Bratu problem (or has no iterate)", i);
            return JFNK_ERR_INVALID_ARG;
        }
        if (p.lv[0].g.n != problems[0]->lv[0].g.n || p.coarse_maxit != problems[0]->coarse_maxit) {
            set_error("jfnk_solve_batched: all hierarchies must end at the same coarse grid");
            return JFNK_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (problems[j] == problems[i]) {
                set_error("jfnk_solve_batched: instance %d repeats a problem object", i);
                return JFNK_ERR_INVALID_ARG;
            }
    }
    BCtx b;
    b.B = count;
    b.o = opts;
    b.st = (cudaStream_t)stream;
    b.lead = problems[0];
    for (int i = 0; i < count; ++i) {
        b.ps.push_back(problems[i]);
        b.u.push_back(u_inout[i]);
    }
    P& lp = *b.lead;
    const size_t res_bytes = ((size_t)count * kResStride * sizeof(double) + 255) & ~size_t(255);
    const size_t dyn_bytes = (size_t)4 << 20;
    if (lp.batch_bytes < res_bytes + dyn_bytes + ((size_t)8 << 20)) {
        set_error("jfnk_solve_batched: staging area too small for %d instances", count);
        return JFNK_ERR_WORKSPACE;
    }
    b.res = reinterpret_cast<double*>(lp.batch);
    b.dyn.dev = lp.batch + res_bytes;
    b.dyn.cap = dyn_bytes;
    b.prog.dev = lp.batch + res_bytes + dyn_bytes;
    b.prog.cap = lp.batch_bytes - res_bytes - dyn_bytes;
    if (lp.pc == JFNK_F32) return bsolve<float>(b, stats);
    return bsolve<double>(b, stats);
}
