// Device building blocks shared by the element-residual kernels: FD-step and
// Chebyshev-coefficient accessors, the per-node epilogues of the fused modes,
// the norm reduction, and the 2D (Bratu) row-segment body used by both the
// single-problem and the batched kernels.
#pragma once
#include "element.cuh"
#include "reduce.cuh"
#include "stencil.cuh"

namespace jfnk {

template <typename T>
__device__ __forceinline__ T eps_of(const EpsSlot* s);
template <>
__device__ __forceinline__ double eps_of<double>(const EpsSlot* s) { return s->e; }
template <>
__device__ __forceinline__ float eps_of<float>(const EpsSlot* s) { return s->ef; }
template <typename T>
__device__ __forceinline__ T inv_eps_of(const EpsSlot* s);
template <>
__device__ __forceinline__ double inv_eps_of<double>(const EpsSlot* s) { return s->inv; }
template <>
__device__ __forceinline__ float inv_eps_of<float>(const EpsSlot* s) { return s->invf; }

template <typename T>
struct ChebK {
    T theta_inv, c1, c2;
};
template <typename T>
__device__ __forceinline__ ChebK<T> cheb_of(const ChebTable* t, int i);
template <>
__device__ __forceinline__ ChebK<double> cheb_of<double>(const ChebTable* t, int i) {
    return {t->theta_inv, t->c1[i], t->c2[i]};
}
template <>
__device__ __forceinline__ ChebK<float> cheb_of<float>(const ChebTable* t, int i) {
    return {t->theta_invf, t->c1f[i], t->c2f[i]};
}

// FP32 square of a value for the norm reductions of the epilogues (the norm
// feeds the FD step and the power-method estimate, which need far less than
// FP32 accuracy).  From FP64 the conversion is done on the integer pipe by
// truncating the significand: on this GPU a hardware FP64 -> FP32 conversion
// runs on the FP64 pipe, the one the FP64 kernels are bound by.  Magnitudes
// below 2^-126 give 0; finite magnitudes beyond the FP32 range saturate to the
// largest finite FP32 value, and a NaN or an infinity gives NaN, so that a
// non-finite result still reaches the FD-step check.
__device__ __forceinline__ float sq_for_norm(float v) { return v * v; }
__device__ __forceinline__ float sq_for_norm(double v) {
    const long long b = __double_as_longlong(v);
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const unsigned int ed = (hi >> 20) & 0x7ffu;
    int e = (int)ed - 1023 + 127;
    unsigned int m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e <= 0) e = 0, m = 0;
    if (e >= 255) e = 254, m = 0x7fffffu;
    if (ed == 0x7ffu) e = 255, m = 0x400000u;  // NaN
    const float f = __int_as_float((int)(((unsigned int)e << 23) | m));
    return f * f;
}

// Per-node epilogue.  val = A(w)_i (already scaled).  Boundary nodes get 0 in
// every output.  `red` accumulates the square of the reduced quantity.
// RAW: val is the unscaled node sum S and A(w)_i = S ns; the FD quotient is
// then formed as S (ns / eps) - A(x)_i / eps with one FMA (ns_inv = ns / eps),
// one FP64 operation fewer per node for the kernels bound by the FP64 pipe.
template <typename T, Mode M, bool RAW = false>
__device__ __forceinline__ void epilogue(const StencilArgs<T>& a, long long idx, bool inner, T val,
                                         T inv_eps, const ChebK<T>& ck, float& red, T ns = T(1),
                                         T ns_inv = T(0)) {
    idx = JFNK_IDX(idx, a.g.size);
    // (A(w)_i - A(x)_i) / eps
    auto fdq = [&](T ax) -> T { return RAW ? fma(val, ns_inv, -(ax * inv_eps)) : (val - ax) * inv_eps; };
    if (M == Mode::F) {
        T f = T(0), av = T(0);
        if (inner) {
            av = RAW ? val * ns : val;
            f = av - (T)a.load_const;
            if (a.load) f -= a.load[idx];
        }
        a.out[idx] = f;
        if (a.out2) a.out2[idx] = av;
        red += sq_for_norm(f);
    } else if (M == Mode::JV) {
        // Au may be F(u) = A(u) - load: the same load is then removed from A(w)
        T jv = T(0);
        if (inner) {
            T base = a.Au[idx] + (T)a.load_const;
            if (a.load) base += a.load[idx];
            jv = fdq(base);
        }
        a.out[idx] = jv;
        red += sq_for_norm(jv);
    } else if (M == Mode::BMJ) {
        T o = inner ? a.rhs[idx] - fdq(a.Au[idx]) : T(0);
        a.out[idx] = o;
        red += sq_for_norm(o);
    } else if (M == Mode::CHEB0) {
        T rr = T(0), dd = T(0);
        if (inner) {
            rr = a.rhs[idx] - fdq(a.Au[idx]);
            dd = rr * ck.theta_inv;
        }
        a.out[idx] = rr;
        a.out2[idx] = dd;
        red += sq_for_norm(dd);
    } else if (M == Mode::CHEB) {
        T rr = T(0), ss = T(0), dn = T(0);
        if (inner) {
            T jd = fdq(a.Au[idx]);
            T dc = a.v[idx];
            rr = a.r[idx] - jd;
            ss = a.s[idx] + dc;
            dn = ck.c1 * dc + ck.c2 * rr;
        }
        a.r[idx] = rr;
        a.s[idx] = ss;
        a.dnew[idx] = dn;
        red += sq_for_norm(dn);
    } else {  // CHEBLAST
        T ss = T(0);
        if (inner) {
            T jd = fdq(a.Au[idx]);
            T dc = a.v[idx];
            T rr = a.r[idx] - jd;
            T dn = ck.c1 * dc + ck.c2 * rr;
            ss = a.s[idx] + dc + dn;
        }
        a.s[idx] = ss;
        red += sq_for_norm(ss);
    }
}

// Epilogue of the adjoint operator: jd = (J^T v)_i at an interior node (0 on
// the boundary); the same fused modes as `epilogue` with J^T v in place of the
// FD action.
template <typename T, Mode M>
__device__ __forceinline__ void epilogue_adj(const StencilArgs<T>& a, long long idx, bool inner, T jd,
                                             const ChebK<T>& ck, float& red) {
    idx = JFNK_IDX(idx, a.g.size);
    if (M == Mode::JV) {
        const T o = inner ? jd : T(0);
        a.out[idx] = o;
        red += sq_for_norm(o);
    } else if (M == Mode::BMJ) {
        const T o = inner ? a.rhs[idx] - jd : T(0);
        a.out[idx] = o;
        red += sq_for_norm(o);
    } else if (M == Mode::CHEB0) {
        T rr = T(0), dd = T(0);
        if (inner) {
            rr = a.rhs[idx] - jd;
            dd = rr * ck.theta_inv;
        }
        a.out[idx] = rr;
        a.out2[idx] = dd;
        red += sq_for_norm(dd);
    } else if (M == Mode::CHEB) {
        T rr = T(0), ss = T(0), dn = T(0);
        if (inner) {
            const T dc = a.v[idx];
            rr = a.r[idx] - jd;
            ss = a.s[idx] + dc;
            dn = ck.c1 * dc + ck.c2 * rr;
        }
        a.r[idx] = rr;
        a.s[idx] = ss;
        a.dnew[idx] = dn;
        red += sq_for_norm(dn);
    } else if (M == Mode::CHEBLAST) {
        T ss = T(0);
        if (inner) {
            const T dc = a.v[idx];
            const T rr = a.r[idx] - jd;
            const T dn = ck.c1 * dc + ck.c2 * rr;
            ss = a.s[idx] + dc + dn;
        }
        a.s[idx] = ss;
        red += sq_for_norm(ss);
    }
}

// bid / nb: index of this CTA among the nb CTAs that reduce together (the
// whole grid, or one instance's CTAs in a batched launch)
template <typename T>
__device__ __forceinline__ void stencil_reduce(const StencilArgs<T>& a, float red, double* sm, unsigned int bid,
                                               unsigned int nb) {
    if (a.red == RedOut::NONE) return;
    double bs = block_sum(red, sm);
    double tot = 0.0;
    if (grid_sum_last_seg(bs, a.partials, a.counter, &tot, sm, bid, nb)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            double nrm = sqrt(tot);
            if (a.red_norm) *a.red_norm = nrm;
            if (a.red == RedOut::EPS || a.red == RedOut::EPS_UNIT)
                set_eps_slot(a.red_eps, a.epsp, nrm, a.red == RedOut::EPS_UNIT, a.status);
        }
    }
}

template <typename T>
__device__ __forceinline__ void stencil_reduce(const StencilArgs<T>& a, float red, double* sm) {
    stencil_reduce(a, red, sm, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                   gridDim.x * gridDim.y * gridDim.z);
}

// Epilogue operands of one node, loaded ahead of the element arithmetic.
template <typename T>
struct EpiIn1 {
    T au, ld, rhs, vv, rr, ss;
};

template <typename T, Mode M>
__device__ __forceinline__ void epi1_load(const StencilArgs<T>& a, long long idx, EpiIn1<T>& e) {
    idx = JFNK_IDX(idx, a.g.size);
    if ((M == Mode::F || M == Mode::JV) && a.load) e.ld = a.load[idx];
    if (M != Mode::F) e.au = a.Au[idx];
    if (M == Mode::BMJ || M == Mode::CHEB0) e.rhs = a.rhs[idx];
    if (M == Mode::CHEB || M == Mode::CHEBLAST) {
        e.vv = a.v[idx];
        e.rr = a.r[idx];
        e.ss = a.s[idx];
    }
}

// `epilogue` (not RAW) with its operands from e: the same operations in the
// same order.
template <typename T, Mode M>
__device__ __forceinline__ void epilogue_pf(const StencilArgs<T>& a, long long idx, bool inner, T val, T inv_eps,
                                            const ChebK<T>& ck, const EpiIn1<T>& e, float& red) {
    idx = JFNK_IDX(idx, a.g.size);
    auto fdq = [&](T ax) -> T { return (val - ax) * inv_eps; };
    if (M == Mode::F) {
        T f = T(0), av = T(0);
        if (inner) {
            av = val;
            f = av - (T)a.load_const;
            if (a.load) f -= e.ld;
        }
        a.out[idx] = f;
        if (a.out2) a.out2[idx] = av;
        red += sq_for_norm(f);
    } else if (M == Mode::JV) {
        T jv = T(0);
        if (inner) {
            T base = e.au + (T)a.load_const;
            if (a.load) base += e.ld;
            jv = fdq(base);
        }
        a.out[idx] = jv;
        red += sq_for_norm(jv);
    } else if (M == Mode::BMJ) {
        T o = inner ? e.rhs - fdq(e.au) : T(0);
        a.out[idx] = o;
        red += sq_for_norm(o);
    } else if (M == Mode::CHEB0) {
        T rr = T(0), dd = T(0);
        if (inner) {
            rr = e.rhs - fdq(e.au);
            dd = rr * ck.theta_inv;
        }
        a.out[idx] = rr;
        a.out2[idx] = dd;
        red += sq_for_norm(dd);
    } else if (M == Mode::CHEB) {
        T rr = T(0), ss = T(0), dn = T(0);
        if (inner) {
            T jd = fdq(e.au);
            T dc = e.vv;
            rr = e.rr - jd;
            ss = e.ss + dc;
            dn = ck.c1 * dc + ck.c2 * rr;
        }
        a.r[idx] = rr;
        a.s[idx] = ss;
        a.dnew[idx] = dn;
        red += sq_for_norm(dn);
    } else {  // CHEBLAST
        T ss = T(0);
        if (inner) {
            T jd = fdq(e.au);
            T dc = e.vv;
            T rr = e.rr - jd;
            T dn = ck.c1 * dc + ck.c2 * rr;
            ss = e.ss + dc + dn;
        }
        a.s[idx] = ss;
        red += sq_for_norm(ss);
    }
}

// ---------------------------------------------------------------------------
// 2D kernel (Bratu), blockDim.x = BX threads, BX-1 output nodes per row segment
// ---------------------------------------------------------------------------
// Row segment [x0, x0+txo) of node rows [y0, y1): blockDim.x = BX >= txo + 1
// threads; smem_raw holds sizeof(T) * (2 (BX+1) + 4 BX) bytes.
template <typename T, Mode M, Prob P = Prob::BRATU2>
__device__ __forceinline__ void stencil2d_body(const StencilArgs<T>& a, int x0, int y0, int y1, int txo,
                                               unsigned int red_bid, unsigned int red_nb, unsigned char* smem_raw,
                                               double* red_sm) {
    const int BX = blockDim.x;
    T* W = reinterpret_cast<T*>(smem_raw);  // [2][BX + 1]
    T* C = W + 2 * (BX + 1);                // [4][BX]
    const int tx = threadIdx.x;
    const Grid g = a.g;
    const int n = g.n;
    T eps = T(0), inv_eps = T(0);
    if (M != Mode::F) {
        eps = eps_of<T>(a.eps);
        inv_eps = inv_eps_of<T>(a.eps);
    }
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    const int ex = x0 - 1 + tx;
    const bool elem_x = tx <= txo && ex >= 0 && ex < n;
    const int nx_o = x0 + tx;
    const bool node_thr = tx < txo && nx_o < g.nx;
    const bool inner_x = nx_o > 0 && nx_o < g.nx - 1;

    // FP32: the next node row is held in registers (u and the masked direction
    // v of this thread's entries i = tx and, where BX = txo + 1, i = tx + BX)
    // from the iteration before it enters the ring, and w = u + eps v is formed
    // when it is stored: no instruction waits on those loads before the element
    // arithmetic.  The epilogue operands of node row j are loaded before the
    // element arithmetic of row j for the same reason.  (Measured: the 4097^2
    // Chebyshev application 12 % and the 64-instance batched solve 6 % faster;
    // in FP64 the extra registers cost 1-4 %, so FP64 loads each row and the
    // epilogue operands where they are used.)
    constexpr bool PF = sizeof(T) == 4;
    auto load_row = [&](int y, int buf) {
        for (int i = tx; i < txo + 2; i += BX) {
            const int x = x0 - 1 + i;
            T val = T(0);
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                const long long idx = JFNK_IDX((long long)y * g.sy + x, g.size);
                val = a.u[idx];
                if (M != Mode::F) {
                    const bool bnd = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1;
                    if (!bnd) val += eps * a.v[idx];
                }
            }
            W[buf * (BX + 1) + i] = val;
        }
    };
    T pu0 = T(0), pv0 = T(0), pu1 = T(0), pv1 = T(0);
    auto load_regs = [&](int y) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = tx + k * BX;
            T uu = T(0), vv = T(0);
            if (i < txo + 2) {
                const int x = x0 - 1 + i;
                if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                    const long long idx = JFNK_IDX((long long)y * g.sy + x, g.size);
                    uu = a.u[idx];
                    if (M != Mode::F) {
                        const bool bnd = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1;
                        if (!bnd) vv = a.v[idx];
                    }
                }
            }
            if (k == 0) {
                pu0 = uu;
                pv0 = vv;
            } else {
                pu1 = uu;
                pv1 = vv;
            }
        }
    };
    auto store_regs = [&](int buf) {
        if (tx < txo + 2) W[buf * (BX + 1) + tx] = (M != Mode::F) ? pu0 + eps * pv0 : pu0;
        if (tx + BX < txo + 2) W[buf * (BX + 1) + tx + BX] = (M != Mode::F) ? pu1 + eps * pv1 : pu1;
    };

    T carry = T(0);
    float red = 0.f;
    if (PF) {
        load_regs(y0 - 1);
        store_regs((y0 - 1) & 1);
        load_regs(y0);
    } else {
        load_row(y0 - 1, (y0 - 1) & 1);
    }
    for (int j = y0 - 1; j < y1; ++j) {
        // row j+1 enters the ring (its slot was last read by row j-1's elements,
        // before the previous iteration's second barrier); row j+2 is loaded
        if (PF) {
            store_regs((j + 1) & 1);
            if (j + 2 <= y1) load_regs(j + 2);
        } else {
            load_row(j + 1, (j + 1) & 1);
        }
        const bool epi = node_thr && j >= y0;
        const long long nidx = (long long)j * g.sy + nx_o;
        EpiIn1<T> e;
        if (PF && epi) epi1_load<T, M>(a, nidx, e);
        __syncthreads();
        T r[4];
        if (elem_x && j >= 0 && j < n) {
            const T* w0 = W + (j & 1) * (BX + 1);
            const T* w1 = W + ((j + 1) & 1) * (BX + 1);
            T ue[4] = {w0[tx], w0[tx + 1], w1[tx], w1[tx + 1]};
            if (P == Prob::MINSURF2)
                elem_minsurf2<T>(ue, a.lh, r);
            else
                elem_bratu2<T>(ue, a.lh, r);
        } else {
            r[0] = r[1] = r[2] = r[3] = T(0);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) C[c * BX + tx] = r[c];
        __syncthreads();
        if (node_thr) {
            const T lower = C[1 * BX + tx] + C[0 * BX + tx + 1];
            const T upper = C[3 * BX + tx] + C[2 * BX + tx + 1];
            if (epi) {
                const bool inner = inner_x && j > 0 && j < g.ny - 1;
                if (PF)
                    epilogue_pf<T, M>(a, nidx, inner, (carry + lower) * a.node_scale, inv_eps, ck, e, red);
                else
                    epilogue<T, M>(a, nidx, inner, (carry + lower) * a.node_scale, inv_eps, ck, red);
            }
            carry = upper;
        }
    }
    stencil_reduce(a, red, red_sm, red_bid, red_nb);
}

}  // namespace jfnk
