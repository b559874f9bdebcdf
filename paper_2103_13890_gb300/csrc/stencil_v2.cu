// 3D element-residual kernel without halo recomputation (grids with n a
// multiple of 32, n >= 64).
//
// A CTA of n x BY threads (n * BY = 1024) owns the elements of BY full x-rows
// [y0, y0+BY) on the layers of one z chunk [z0, z1): every element of the grid
// is evaluated exactly once and every warp is full.  Thread (x, w) evaluates the
// element with lower corner (x, y0+w, k) on each layer k; node planes live in a
// three-plane shared ring (the plane after next is prefetched into registers
// while the current layer is computed) and the element contributions are
// exchanged through shared memory.  A node's total is
//     lo(layer k) + hi(layer k-1),
// summed over the 2^2 elements around it in the xy plane in a fixed order; the
// hi part is carried in a register from one layer to the next.
//
// Nodes on internal tile faces -- the node rows y0 and y0+BY shared with the
// neighbouring y tiles and the planes z0 and z1 shared with the neighbouring z
// chunks -- receive only part of their element contributions in this CTA.  The
// CTA stores those partial sums in a face buffer, and stencil3d_fixup_kernel
// adds the two (four on an edge) partials in a fixed order and applies the same
// epilogue.  The fixup kernel also completes the norm reduction, so results are
// deterministic.  Every F_i is still the sum of the same element integrals.
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "element.cuh"
#include "pf2.cuh"
#include "reduce.cuh"
#include "stencil.cuh"
#include "stencil_v2.cuh"

// face-buffer index, checked against the buffer in bounds-checked builds
#define JFNK_IDX_FACE(i) JFNK_IDX((i), a.face_cap)

namespace jfnk {

// Bit of the current device in a per-kernel mask of devices whose function
// attributes are set (function attributes are set per device).  Ordinals from
// 63 up get no bit and set the attributes at every launch.
static unsigned long long device_bit() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 63) return 0;
    return 1ull << dev;
}

template <typename T>
__device__ __forceinline__ T eps_of2(const EpsSlot* s);
template <>
__device__ __forceinline__ double eps_of2<double>(const EpsSlot* s) { return s->e; }
template <>
__device__ __forceinline__ float eps_of2<float>(const EpsSlot* s) { return s->ef; }
template <typename T>
__device__ __forceinline__ T inv_eps_of2(const EpsSlot* s);
template <>
__device__ __forceinline__ double inv_eps_of2<double>(const EpsSlot* s) { return s->inv; }
template <>
__device__ __forceinline__ float inv_eps_of2<float>(const EpsSlot* s) { return s->invf; }

template <typename T>
struct ChebK2 {
    T theta_inv, c1, c2;
};
template <typename T>
__device__ __forceinline__ ChebK2<T> cheb_of2(const ChebTable* t, int i);
template <>
__device__ __forceinline__ ChebK2<double> cheb_of2<double>(const ChebTable* t, int i) {
    return {t->theta_inv, t->c1[i], t->c2[i]};
}
template <>
__device__ __forceinline__ ChebK2<float> cheb_of2<float>(const ChebTable* t, int i) {
    return {t->theta_invf, t->c1f[i], t->c2f[i]};
}

// Per-node epilogue (same definitions as the tiled kernel's): val = A(w)_i.
template <typename T, Mode M>
__device__ __forceinline__ void epilogue2(const StencilArgs<T>& a, int idx, bool inner, T val, T inv_eps,
                                          const ChebK2<T>& ck, float& red) {
    idx = (int)JFNK_IDX(idx, a.g.size);
    if (M == Mode::F) {
        T f = T(0), av = T(0);
        if (inner) {
            av = val;
            f = val - (T)a.load_const;
            if (a.load) f -= a.load[idx];
        }
        a.out[idx] = f;
        if (a.out2) a.out2[idx] = av;
        red += (float)f * (float)f;
    } else if (M == Mode::JV) {
        T jv = T(0);
        if (inner) {
            T aw = val - (T)a.load_const;
            if (a.load) aw -= a.load[idx];
            jv = (aw - a.Au[idx]) * inv_eps;
        }
        a.out[idx] = jv;
        red += (float)jv * (float)jv;
    } else if (M == Mode::BMJ) {
        T o = inner ? a.rhs[idx] - (val - a.Au[idx]) * inv_eps : T(0);
        a.out[idx] = o;
        red += (float)o * (float)o;
    } else if (M == Mode::CHEB0) {
        T rr = T(0), dd = T(0);
        if (inner) {
            rr = a.rhs[idx] - (val - a.Au[idx]) * inv_eps;
            dd = rr * ck.theta_inv;
        }
        a.out[idx] = rr;
        a.out2[idx] = dd;
        red += (float)dd * (float)dd;
    } else if (M == Mode::CHEB) {
        T rr = T(0), ss = T(0), dn = T(0);
        if (inner) {
            T jd = (val - a.Au[idx]) * inv_eps;
            T dc = a.v[idx];
            rr = a.r[idx] - jd;
            ss = a.s[idx] + dc;
            dn = ck.c1 * dc + ck.c2 * rr;
        }
        a.r[idx] = rr;
        a.s[idx] = ss;
        a.dnew[idx] = dn;
        red += (float)dn * (float)dn;
    } else {  // CHEBLAST
        T ss = T(0);
        if (inner) {
            T jd = (val - a.Au[idx]) * inv_eps;
            T dc = a.v[idx];
            T rr = a.r[idx] - jd;
            T dn = ck.c1 * dc + ck.c2 * rr;
            ss = a.s[idx] + dc + dn;
        }
        a.s[idx] = ss;
        red += (float)ss * (float)ss;
    }
}

// Epilogue operands of one node, loaded at the start of a layer so that their
// latency overlaps the element arithmetic.
template <typename T>
struct EpiIn {
    T au, vv, rr, ss, rhs, ld;
};

template <typename T, Mode M>
__device__ __forceinline__ void epi_load(const StencilArgs<T>& a, int idx, EpiIn<T>& e) {
    if (M == Mode::F || M == Mode::JV) e.ld = a.load ? a.load[idx] : T(0);
    if (M != Mode::F) e.au = a.Au[idx];
    if (M == Mode::BMJ || M == Mode::CHEB0) e.rhs = a.rhs[idx];
    if (M == Mode::CHEB || M == Mode::CHEBLAST) {
        e.vv = a.v[idx];
        e.rr = a.r[idx];
        e.ss = a.s[idx];
    }
}

// Same definitions as epilogue2 for an interior node, operands from e.
template <typename T, Mode M>
__device__ __forceinline__ void epilogue2_pf(const StencilArgs<T>& a, int idx, T val, T inv_eps,
                                             const ChebK2<T>& ck, const EpiIn<T>& e, float& red) {
    idx = (int)JFNK_IDX(idx, a.g.size - 1);
    if (M == Mode::F) {
        const T f = val - (T)a.load_const - e.ld;
        a.out[idx] = f;
        if (a.out2) a.out2[idx] = val;
        red += (float)f * (float)f;
    } else if (M == Mode::JV) {
        const T jv = (val - (T)a.load_const - e.ld - e.au) * inv_eps;
        a.out[idx] = jv;
        red += (float)jv * (float)jv;
    } else if (M == Mode::BMJ) {
        const T o = e.rhs - (val - e.au) * inv_eps;
        a.out[idx] = o;
        red += (float)o * (float)o;
    } else if (M == Mode::CHEB0) {
        const T rr = e.rhs - (val - e.au) * inv_eps;
        const T dd = rr * ck.theta_inv;
        a.out[idx] = rr;
        a.out2[idx] = dd;
        red += (float)dd * (float)dd;
    } else if (M == Mode::CHEB) {
        const T jd = (val - e.au) * inv_eps;
        const T rr = e.rr - jd;
        const T dn = ck.c1 * e.vv + ck.c2 * rr;
        a.r[idx] = rr;
        a.s[idx] = e.ss + e.vv;
        a.dnew[idx] = dn;
        red += (float)dn * (float)dn;
    } else {
        const T jd = (val - e.au) * inv_eps;
        const T rr = e.rr - jd;
        const T dn = ck.c1 * e.vv + ck.c2 * rr;
        const T ss = e.ss + e.vv + dn;
        a.s[idx] = ss;
        red += (float)ss * (float)ss;
    }
}

// Face buffer addressing
__device__ __forceinline__ int ylo_idx(const V2Geom& q, int ty, int c, int zl, int x) {
    return (int)q.ylo + (((int)ty * q.Tz + c) * (q.ZC + 1) + zl) * (q.n + 1) + x;
}
__device__ __forceinline__ int yhi_idx(const V2Geom& q, int ty, int c, int zl, int x) {
    return (int)q.yhi + (((int)ty * q.Tz + c) * (q.ZC + 1) + zl) * (q.n + 1) + x;
}
__device__ __forceinline__ int zlo_idx(const V2Geom& q, int ty, int c, int w, int x) {
    return (int)q.zlo + (((int)ty * q.Tz + c) * (q.BY + 1) + w) * (q.n + 1) + x;
}
__device__ __forceinline__ int zhi_idx(const V2Geom& q, int ty, int c, int w, int x) {
    return (int)q.zhi + (((int)ty * q.Tz + c) * (q.BY + 1) + w) * (q.n + 1) + x;
}

template <typename T, Prob P, Mode M>
__global__ void __launch_bounds__(kV2Threads, 1) stencil3d_v2_kernel(const StencilArgs<T> a, const V2Geom q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = q.n, BY = q.BY, NP = n + 1;
    T* W = reinterpret_cast<T*>(smem_raw);  // [3][BY+1][n+1]
    T* C2 = W + 3 * (BY + 1) * NP;          // [2][8][BY][n] (double-buffered by layer parity)
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int sy32 = (int)g.sy, sz32 = (int)g.sz;  // (n+1)^3 < 2^31 for n <= 512
    const int tx = threadIdx.x, w = threadIdx.y;
    const int ty = blockIdx.x, c = blockIdx.y;
    const int y0 = ty * BY;
    const int z0 = c * q.ZC;
    const int z1 = min(z0 + q.ZC, n);
    T eps = T(0), inv_eps = T(0);
    if (M != Mode::F) {
        eps = eps_of2<T>(a.eps);
        inv_eps = inv_eps_of2<T>(a.eps);
    }
    ChebK2<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of2<T>(a.cheb, a.cheb_step);

    // nodal value of w = x + eps v at (x, y, z); boundary entries of v ignored
    auto node_val = [&](int x, int y, int z) -> T {
        const int idx = (int)JFNK_IDX((int)z * sz32 + (int)y * sy32 + x, g.size);
        T val = a.u[idx];
        if (M != Mode::F) {
            const bool bnd = x == 0 || x == n || y == 0 || y == n || z == 0 || z == n;
            if (!bnd) val += eps * a.v[idx];
        }
        return val;
    };
    // this thread's share of a plane: (tx, y0+w); row y0+BY (w == 0); column n (tx == n-1)
    const bool extra_row = (w == 0);
    const bool extra_col = (tx == n - 1);
    auto load4 = [&](int z, T& p0, T& p1, T& p2, T& p3) {
        p0 = node_val(tx, y0 + w, z);
        if (extra_col) p1 = node_val(n, y0 + w, z);
        if (extra_row) p2 = node_val(tx, y0 + BY, z);
        if (extra_row && extra_col) p3 = node_val(n, y0 + BY, z);
    };
    auto store4 = [&](int buf, T p0, T p1, T p2, T p3) {
        T* Wb = W + buf * (BY + 1) * NP;
        Wb[w * NP + tx] = p0;
        if (extra_col) Wb[w * NP + n] = p1;
        if (extra_row) Wb[BY * NP + tx] = p2;
        if (extra_row && extra_col) Wb[BY * NP + n] = p3;
    };

    T q0 = T(0), q1 = T(0), q2 = T(0), q3 = T(0);
    load4(z0, q0, q1, q2, q3);
    store4(z0 % 3, q0, q1, q2, q3);
    load4(z0 + 1, q0, q1, q2, q3);
    store4((z0 + 1) % 3, q0, q1, q2, q3);
    __syncthreads();

    // rows handled by this thread: own row y0+w, and for w == 0 also row y0+BY
    const int yA = y0 + w, yB = y0 + BY;
    const bool faceA = (w == 0) && y0 > 0;         // shared with the tile below
    const bool bndA = (yA == 0);
    const bool bndB = yB == n;
    T carryA = T(0), carryB = T(0);
    float red = 0.f;
    const T scale = a.node_scale;
    const T zero = T(0);
    const ChebK2<T> ck0 = ck;

    for (int k = z0; k < z1; ++k) {
        T* C = C2 + (k & 1) * 8 * BY * n;
        const bool pf = (k + 2 <= z1);
        if (pf) load4(k + 2, q0, q1, q2, q3);
        // operands of the node epilogue of this layer (complete nodes only)
        const int idxA = (int)k * sz32 + (int)yA * sy32 + tx;
        const bool completeA = !(k == 0 || bndA || tx == 0 || faceA || k == z0);
        EpiIn<T> eA;
        if (completeA) epi_load<T, M>(a, idxA, eA);
        const T* W0 = W + (k % 3) * (BY + 1) * NP;
        const T* W1 = W + ((k + 1) % 3) * (BY + 1) * NP;
        T ue[8] = {W0[w * NP + tx],       W0[w * NP + tx + 1],       W0[(w + 1) * NP + tx],
                   W0[(w + 1) * NP + tx + 1], W1[w * NP + tx],       W1[w * NP + tx + 1],
                   W1[(w + 1) * NP + tx],     W1[(w + 1) * NP + tx + 1]};
        T r[8];
        if (P == Prob::NDK3)
            elem_nd3<T, true>(ue, a.kappa[((int)k * n + (y0 + w)) * n + tx], r);
        else
            elem_nd3<T, false>(ue, T(1), r);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) C[(cc * BY + w) * n + tx] = r[cc];
        // the ring slot of plane k+2 was last read by layer k-1 (before the
        // previous barrier); the barrier below publishes it for layer k+1
        if (pf) store4((k + 2) % 3, q0, q1, q2, q3);
        __syncthreads();
        // own row y0+w: b = 0 corners of row w, b = 1 corners of row w-1
        T loA = C[(0 * BY + w) * n + tx];
        T hiA = C[(4 * BY + w) * n + tx];
        if (tx > 0) {
            loA += C[(1 * BY + w) * n + tx - 1];
            hiA += C[(5 * BY + w) * n + tx - 1];
        }
        if (w > 0) {
            loA += C[(2 * BY + w - 1) * n + tx];
            hiA += C[(6 * BY + w - 1) * n + tx];
            if (tx > 0) {
                loA += C[(3 * BY + w - 1) * n + tx - 1];
                hiA += C[(7 * BY + w - 1) * n + tx - 1];
            }
        }
        T loB = T(0), hiB = T(0);
        if (extra_row) {  // row y0+BY: b = 1 corners of row BY-1
            loB = C[(2 * BY + BY - 1) * n + tx];
            hiB = C[(6 * BY + BY - 1) * n + tx];
            if (tx > 0) {
                loB += C[(3 * BY + BY - 1) * n + tx - 1];
                hiB += C[(7 * BY + BY - 1) * n + tx - 1];
            }
        }
        // plane k
        {
            const T vA = loA + carryA;
            const int idx = (int)k * sz32 + (int)yA * sy32 + tx;
            if (k == 0 || bndA || tx == 0) {
                epilogue2<T, M>(a, idx, false, zero, inv_eps, ck0, red);
            } else if (faceA) {
                a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, k - z0, tx))] = vA;
            } else if (k == z0) {
                a.face[JFNK_IDX_FACE(zlo_idx(q, ty, c, w, tx))] = vA;
            } else {
                epilogue2_pf<T, M>(a, idx, vA * scale, inv_eps, ck0, eA, red);
            }
            if (extra_col) epilogue2<T, M>(a, idx + 1, false, zero, inv_eps, ck0, red);  // x = n
            carryA = hiA;
        }
        if (extra_row) {
            const T vB = loB + carryB;
            const int idx = (int)k * sz32 + (int)yB * sy32 + tx;
            if (k == 0 || bndB || tx == 0) {
                epilogue2<T, M>(a, idx, false, zero, inv_eps, ck0, red);
            } else {
                a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, k - z0, tx))] = vB;
            }
            if (extra_col) epilogue2<T, M>(a, idx + 1, false, zero, inv_eps, ck0, red);
            carryB = hiB;
        }
    }
    // plane z1: the carries are partial sums from the last layer only
    {
        const int idx = (int)z1 * sz32 + (int)yA * sy32 + tx;
        if (z1 == n || bndA || tx == 0) {
            epilogue2<T, M>(a, idx, false, zero, inv_eps, ck0, red);
        } else if (faceA) {
            a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, z1 - z0, tx))] = carryA;
        } else {
            a.face[JFNK_IDX_FACE(zhi_idx(q, ty, c, w, tx))] = carryA;
        }
        if (extra_col) epilogue2<T, M>(a, idx + 1, false, zero, inv_eps, ck0, red);
        if (extra_row) {
            const int idxB = (int)z1 * sz32 + (int)yB * sy32 + tx;
            if (z1 == n || bndB || tx == 0) {
                epilogue2<T, M>(a, idxB, false, zero, inv_eps, ck0, red);
            } else {
                a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, z1 - z0, tx))] = carryB;
            }
            if (extra_col) epilogue2<T, M>(a, idxB + 1, false, zero, inv_eps, ck0, red);
        }
    }
    // block partial of the norm; the fixup kernel completes the reduction
    if (a.red != RedOut::NONE) {
        const double bs = block_sum(red, red_sm);
        if (threadIdx.x == 0 && threadIdx.y == 0) a.partials[blockIdx.x + gridDim.x * blockIdx.y] = bs;
    }
}

// ---------------------------------------------------------------------------
// FP32 variant with two elements per thread.  Thread (t, w) of an (n/2) x BY
// CTA owns the elements with lower corners (2t, y0+w, k) and (2t+1, y0+w, k)
// and evaluates both at once in the packed f32x2 form (pf2.cuh): the element
// routine, the node-plane ring, the layer loop, the node totals and the face
// buffer are those of the kernel above (same tiling, same fixup), with half
// the threads and half the instructions per element.  Node rows in shared
// memory have an even pitch, so the pair (2t, 2t+1) is one 8-byte word, and
// the contributions of the corners with a = 1 (those to node x+1 of element
// x) are stored one place to the right, so that the node pair (2t, 2t+1)
// reads every corner of its 2^2 in-plane elements as one aligned pair.  The
// per-node sums are added in the same order as above.  MINB: the CTAs per SM
// the launch bounds provide for (1: up to 128 registers a thread, 2: 64).
// ---------------------------------------------------------------------------
template <Prob P, Mode M, int MINB>
__global__ void __launch_bounds__(kV3Threads, MINB) stencil3d_v3_kernel(const StencilArgs<float> a, const V2Geom q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = q.n, BY = q.BY, NP = n + 2;
    float* W = reinterpret_cast<float*>(smem_raw);  // [3][BY+1][NP]
    float* C2 = W + 3 * (BY + 1) * NP;              // [2][8][BY][NP] (double-buffered by layer parity)
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int sy32 = (int)g.sy, sz32 = (int)g.sz;
    const int t = threadIdx.x, w = threadIdx.y;
    const int x0 = 2 * t;
    const int ty = blockIdx.x, c = blockIdx.y;
    const int y0 = ty * BY;
    const int z0 = c * q.ZC;
    const int z1 = min(z0 + q.ZC, n);
    float eps = 0.f, inv_eps = 0.f;
    if (M != Mode::F) {
        eps = eps_of2<float>(a.eps);
        inv_eps = inv_eps_of2<float>(a.eps);
    }
    ChebK2<float> ck = {0.f, 0.f, 0.f};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of2<float>(a.cheb, a.cheb_step);

    // u and the masked direction v (0 on the boundary) of node (x, y, z); w = u +
    // eps v is formed when the plane is stored, so that no instruction waits on
    // the loads before the layer's element arithmetic
    auto node_uv = [&](int x, int y, int z, float& uu, float& vv) {
        const int idx = (int)JFNK_IDX(z * sz32 + y * sy32 + x, g.size);
        uu = a.u[idx];
        vv = 0.f;
        if (M != Mode::F) {
            const bool bnd = x == 0 || x == n || y == 0 || y == n || z == 0 || z == n;
            if (!bnd) vv = a.v[idx];
        }
    };
    // this thread's share of a plane: nodes (2t, 2t+1) of row y0+w, of row
    // y0+BY (w == 0), and node n of those rows (last t)
    const bool extra_row = (w == 0);
    const bool extra_col = (x0 == n - 2);
    // the next plane in registers (u in p, v in q): loaded at the start of a
    // layer, stored to the ring after the layer's element arithmetic
    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f, p5 = 0.f;
    float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 0.f;
    auto load_plane = [&](int z) {
        node_uv(x0, y0 + w, z, p0, q0);
        node_uv(x0 + 1, y0 + w, z, p1, q1);
        if (extra_col) node_uv(n, y0 + w, z, p2, q2);
        if (extra_row) {
            node_uv(x0, y0 + BY, z, p3, q3);
            node_uv(x0 + 1, y0 + BY, z, p4, q4);
        }
        if (extra_row && extra_col) node_uv(n, y0 + BY, z, p5, q5);
    };
    auto wv = [&](float uu, float vv) { return M != Mode::F ? uu + eps * vv : uu; };
    auto store_plane = [&](int buf) {
        float* Wb = W + buf * (BY + 1) * NP;
        pf2_store(Wb + w * NP + x0, pf2_pack(wv(p0, q0), wv(p1, q1)));
        if (extra_col) Wb[w * NP + n] = wv(p2, q2);
        if (extra_row) pf2_store(Wb + BY * NP + x0, pf2_pack(wv(p3, q3), wv(p4, q4)));
        if (extra_row && extra_col) Wb[BY * NP + n] = wv(p5, q5);
    };

    load_plane(z0);
    store_plane(z0 % 3);
    load_plane(z0 + 1);
    store_plane((z0 + 1) % 3);

    if (t == 0) {  // node 0 has no element on its left: its shifted a = 1 slots stay 0
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int cc = 1; cc < 8; cc += 2) C2[((b * 8 + cc) * BY + w) * NP] = 0.f;
    }
    __syncthreads();

    const int yA = y0 + w, yB = y0 + BY;
    const bool faceA = (w == 0) && y0 > 0;  // shared with the tile below
    const bool bndA = (yA == 0);
    const bool bndB = yB == n;
    pf2 carryA = pf2(0.0), carryB = pf2(0.0);
    float red = 0.f;
    const float scale = a.node_scale;
    const ChebK2<float> ck0 = ck;
    auto zero_node = [&](int idx) { epilogue2<float, M>(a, idx, false, 0.f, inv_eps, ck0, red); };

    for (int k = z0; k < z1; ++k) {
        float* C = C2 + (k & 1) * 8 * BY * NP;
        const bool pf = (k + 2 <= z1);
        if (pf) load_plane(k + 2);
        // operands of this layer's node epilogue (complete nodes of row yA only)
        const int idxA = k * sz32 + yA * sy32 + x0;
        const bool rowComplete = !(k == 0 || bndA || faceA || k == z0);
        EpiIn<float> e0, e1;
        if (rowComplete && x0 > 0) epi_load<float, M>(a, idxA, e0);
        if (rowComplete) epi_load<float, M>(a, idxA + 1, e1);
        // corners of the element pair: a = 0 -> nodes (2t, 2t+1), a = 1 -> nodes (2t+1, 2t+2)
        const float* W0 = W + (k % 3) * (BY + 1) * NP;
        const float* W1 = W + ((k + 1) % 3) * (BY + 1) * NP;
        pf2 ue[8];
        {
            const float* rows[4] = {W0 + w * NP + x0, W0 + (w + 1) * NP + x0, W1 + w * NP + x0,
                                    W1 + (w + 1) * NP + x0};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ue[2 * i] = pf2_load(rows[i]);
                float lo, hi;
                pf2_unpack(ue[2 * i], lo, hi);
                ue[2 * i + 1] = pf2_pack(hi, rows[i][2]);
            }
        }
        pf2 r[8];
        if (P == Prob::NDK3)
            elem_nd3<pf2, true>(ue, pf2_load(a.kappa + (k * n + yA) * n + x0), r);
        else
            elem_nd3<pf2, false>(ue, pf2(1.0), r);
        float* Cw = C + w * NP + x0;
#pragma unroll
        for (int cc = 0; cc < 8; cc += 2) pf2_store(Cw + cc * BY * NP, r[cc]);
#pragma unroll
        for (int cc = 1; cc < 8; cc += 2) {
            float lo, hi;
            pf2_unpack(r[cc], lo, hi);
            Cw[cc * BY * NP + 1] = lo;
            Cw[cc * BY * NP + 2] = hi;
        }
        // the ring slot of plane k+2 was last read by layer k-1 (before the
        // previous barrier); the barrier below publishes it for layer k+1
        if (pf) store_plane((k + 2) % 3);
        __syncthreads();
        // own row y0+w: b = 0 corners of element row w, b = 1 corners of row w-1
        pf2 loA = pf2_load(Cw) + pf2_load(Cw + 1 * BY * NP);
        pf2 hiA = pf2_load(Cw + 4 * BY * NP) + pf2_load(Cw + 5 * BY * NP);
        if (w > 0) {
            loA = loA + pf2_load(Cw + 2 * BY * NP - NP);
            hiA = hiA + pf2_load(Cw + 6 * BY * NP - NP);
            loA = loA + pf2_load(Cw + 3 * BY * NP - NP);
            hiA = hiA + pf2_load(Cw + 7 * BY * NP - NP);
        }
        pf2 loB = pf2(0.0), hiB = pf2(0.0);
        if (extra_row) {  // row y0+BY: b = 1 corners of element row BY-1
            const float* Cb = C + (BY - 1) * NP + x0;
            loB = pf2_load(Cb + 2 * BY * NP) + pf2_load(Cb + 3 * BY * NP);
            hiB = pf2_load(Cb + 6 * BY * NP) + pf2_load(Cb + 7 * BY * NP);
        }
        // plane k
        {
            float v0, v1;
            pf2_unpack(loA + carryA, v0, v1);
            if (k == 0 || bndA) {
                zero_node(idxA);
                zero_node(idxA + 1);
            } else if (faceA) {
                if (x0 == 0) zero_node(idxA);
                else a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, k - z0, x0))] = v0;
                a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, k - z0, x0 + 1))] = v1;
            } else if (k == z0) {
                if (x0 == 0) zero_node(idxA);
                else a.face[JFNK_IDX_FACE(zlo_idx(q, ty, c, w, x0))] = v0;
                a.face[JFNK_IDX_FACE(zlo_idx(q, ty, c, w, x0 + 1))] = v1;
            } else {
                if (x0 == 0) zero_node(idxA);
                else epilogue2_pf<float, M>(a, idxA, v0 * scale, inv_eps, ck0, e0, red);
                epilogue2_pf<float, M>(a, idxA + 1, v1 * scale, inv_eps, ck0, e1, red);
            }
            if (extra_col) zero_node(idxA + 2);  // x = n
            carryA = hiA;
        }
        if (extra_row) {
            float v0, v1;
            pf2_unpack(loB + carryB, v0, v1);
            const int idx = k * sz32 + yB * sy32 + x0;
            if (k == 0 || bndB) {
                zero_node(idx);
                zero_node(idx + 1);
            } else {
                if (x0 == 0) zero_node(idx);
                else a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, k - z0, x0))] = v0;
                a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, k - z0, x0 + 1))] = v1;
            }
            if (extra_col) zero_node(idx + 2);
            carryB = hiB;
        }
    }
    // plane z1: the carries are partial sums from the last layer only
    {
        float v0, v1;
        pf2_unpack(carryA, v0, v1);
        const int idx = z1 * sz32 + yA * sy32 + x0;
        if (z1 == n || bndA) {
            zero_node(idx);
            zero_node(idx + 1);
        } else if (faceA) {
            if (x0 == 0) zero_node(idx);
            else a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, z1 - z0, x0))] = v0;
            a.face[JFNK_IDX_FACE(ylo_idx(q, ty, c, z1 - z0, x0 + 1))] = v1;
        } else {
            if (x0 == 0) zero_node(idx);
            else a.face[JFNK_IDX_FACE(zhi_idx(q, ty, c, w, x0))] = v0;
            a.face[JFNK_IDX_FACE(zhi_idx(q, ty, c, w, x0 + 1))] = v1;
        }
        if (extra_col) zero_node(idx + 2);
        if (extra_row) {
            pf2_unpack(carryB, v0, v1);
            const int idxB = z1 * sz32 + yB * sy32 + x0;
            if (z1 == n || bndB) {
                zero_node(idxB);
                zero_node(idxB + 1);
            } else {
                if (x0 == 0) zero_node(idxB);
                else a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, z1 - z0, x0))] = v0;
                a.face[JFNK_IDX_FACE(yhi_idx(q, ty, c, z1 - z0, x0 + 1))] = v1;
            }
            if (extra_col) zero_node(idxB + 2);
        }
    }
    if (a.red != RedOut::NONE) {
        const double bs = block_sum(red, red_sm);
        if (threadIdx.x == 0 && threadIdx.y == 0) a.partials[blockIdx.x + gridDim.x * blockIdx.y] = bs;
    }
}

template <typename T, Mode M>
__global__ void __launch_bounds__(256) stencil3d_fixup_kernel(const StencilArgs<T> a, const V2Geom q, int main_blocks) {
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int sy32 = (int)g.sy, sz32 = (int)g.sz;
    const int n = q.n, BY = q.BY, ZC = q.ZC;
    const int m1 = n - 1;
    const int countA = (int)(q.Ty - 1) * m1 * m1;
    const int rowsB = m1 - (q.Ty - 1);
    const int countB = (int)(q.Tz - 1) * rowsB * m1;
    T inv_eps = T(0);
    if (M != Mode::F) inv_eps = inv_eps_of2<T>(a.eps);
    ChebK2<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of2<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    for (int i = blockIdx.x * (int)blockDim.x + threadIdx.x; i < countA + countB;
         i += (int)gridDim.x * blockDim.x) {
        int x, y, z;
        T total;
        if (i < countA) {
            const int tyb = (int)(i / (m1 * m1)) + 1;
            const int rem = i % (m1 * m1);
            z = (int)(rem / m1) + 1;
            x = (int)(rem % m1) + 1;
            y = tyb * BY;
            const int cz = z / ZC, zl = z - cz * ZC;
            if (zl != 0) {
                total = a.face[JFNK_IDX_FACE(yhi_idx(q, tyb - 1, cz, zl, x))] + a.face[JFNK_IDX_FACE(ylo_idx(q, tyb, cz, zl, x))];
            } else {
                total = (a.face[JFNK_IDX_FACE(yhi_idx(q, tyb - 1, cz - 1, ZC, x))] + a.face[JFNK_IDX_FACE(ylo_idx(q, tyb, cz - 1, ZC, x))]) +
                        (a.face[JFNK_IDX_FACE(yhi_idx(q, tyb - 1, cz, 0, x))] + a.face[JFNK_IDX_FACE(ylo_idx(q, tyb, cz, 0, x))]);
            }
        } else {
            const int j = i - countA;
            const int cb = (int)(j / (rowsB * m1)) + 1;
            const int rem = j % (rowsB * m1);
            const int yi = (int)(rem / m1);
            x = (int)(rem % m1) + 1;
            y = (yi / (BY - 1)) * BY + (yi % (BY - 1)) + 1;
            z = cb * ZC;
            const int tyy = y / BY, ww = y - tyy * BY;
            total = a.face[JFNK_IDX_FACE(zhi_idx(q, tyy, cb - 1, ww, x))] + a.face[JFNK_IDX_FACE(zlo_idx(q, tyy, cb, ww, x))];
        }
        const int idx = (int)z * sz32 + (int)y * sy32 + x;
        epilogue2<T, M>(a, idx, true, total * a.node_scale, inv_eps, ck, red);
    }
    if (a.red == RedOut::NONE) return;
    const double bs = block_sum(red, red_sm);
    __shared__ int s_last;
    const int tid = threadIdx.x;
    if (tid == 0) {
        a.partials[main_blocks + blockIdx.x] = bs;
        __threadfence();
        const unsigned int prev = atomicAdd(a.counter, 1u);
        s_last = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int total_blocks = main_blocks + gridDim.x;
    double s = 0.0;
    for (int b = tid; b < total_blocks; b += blockDim.x) s += __ldcg(&a.partials[b]);
    s = block_sum(s, red_sm);
    if (tid == 0) {
        *a.counter = 0u;
        const double nrm = sqrt(s);
        if (a.red_norm) *a.red_norm = nrm;
        if (a.red == RedOut::EPS || a.red == RedOut::EPS_UNIT)
            set_eps_slot(a.red_eps, a.epsp, nrm, a.red == RedOut::EPS_UNIT, a.status);
    }
}

// ---------------------------------------------------------------------------
bool v2_applicable(const Grid& g) {
    return g.d == 3 && !g.beam && g.n >= 64 && g.n <= 512 && (g.n % 32) == 0;
}

V2Geom v2_geometry(const Grid& g, int num_sms, int max_threads) {
    V2Geom q;
    q.n = g.n;
    if (max_threads <= 0 || max_threads > kV2Threads) max_threads = kV2Threads;
    // rows per CTA: the largest divisor of n with n * BY <= max_threads, so that
    // the y tiles cover all n element rows exactly
    q.BY = std::max(1, max_threads / g.n);
    while (q.BY > 1 && g.n % q.BY != 0) --q.BY;
    q.Ty = g.n / q.BY;
    // z chunks: minimise waves x layers per CTA over whole waves of the CTAs an SM holds
    num_sms *= std::max(1, kV2Threads / (g.n * q.BY));
    int best_tz = 1;
    long long best_cost = -1;
    for (int tz = 1; tz <= g.n; ++tz) {
        const int zc = (g.n + tz - 1) / tz;
        if ((long long)(tz - 1) * zc >= g.n) continue;  // no empty chunk
        // the block partials of the main and fixup kernels share 2 kMaxRedBlocks slots
        if (tz > 1 && (long long)q.Ty * tz > 2 * kMaxRedBlocks - 4 * kNumSMs) break;
        const long long waves = ((long long)q.Ty * tz + num_sms - 1) / num_sms;
        const long long cost = waves * (zc + 1) * 16 + (tz - 1);  // small preference for fewer faces
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_tz = tz;
        }
    }
    q.Tz = best_tz;
    q.ZC = (g.n + q.Tz - 1) / q.Tz;
    const long long ysz = (long long)q.Ty * q.Tz * (q.ZC + 1) * (q.n + 1);
    const long long zsz = (long long)q.Ty * q.Tz * (q.BY + 1) * (q.n + 1);
    q.ylo = 0;
    q.yhi = ysz;
    q.zlo = 2 * ysz;
    q.zhi = 2 * ysz + zsz;
    q.face_count = 2 * ysz + 2 * zsz;
    return q;
}

long long v2_face_count(const Grid& g, int max_threads) {
    if (!v2_applicable(g)) return 0;
    return v2_geometry(g, kNumSMs, max_threads).face_count;
}

static int fixup_blocks(const V2Geom& q) {
    const long long m1 = q.n - 1;
    const long long cnt = (long long)(q.Ty - 1) * m1 * m1 + (long long)(q.Tz - 1) * (m1 - (q.Ty - 1)) * m1;
    long long b = (cnt + 255) / 256;
    if (b > 4 * kNumSMs) b = 4 * kNumSMs;
    return (int)(b < 1 ? 1 : b);
}

template <typename T, Prob P, Mode M>
static jfnk_status launch_v2_pm(const StencilArgs<T>& a, cudaStream_t st) {
    const V2Geom q = v2_geometry(a.g, kNumSMs, a.v2_threads);
    if (q.face_count > a.face_cap) {
        set_error("face scratch too small (%lld < %lld)", a.face_cap, q.face_count);
        return JFNK_ERR_WORKSPACE;
    }
    const int main_blocks = q.Ty * q.Tz;
    const int fb = fixup_blocks(q);
    if (main_blocks + fb > kMaxRedBlocks * 2) {
        set_error("v2 grid too large for the reduction scratch");
        return JFNK_ERR_INVALID_ARG;
    }
    const size_t smem = sizeof(T) * (3 * (size_t)(q.BY + 1) * (q.n + 1) + 16 * (size_t)q.BY * q.n);
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose attribute is set
    const unsigned long long dbit = device_bit();
    if (!(attr_devs.load() & dbit)) {
        JFNK_CUDA_TRY(cudaFuncSetAttribute(stencil3d_v2_kernel<T, P, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           220 * 1024));
        attr_devs.fetch_or(dbit);
    }
    stencil3d_v2_kernel<T, P, M><<<dim3(q.Ty, q.Tz), dim3(q.n, q.BY), smem, st>>>(a, q);
    JFNK_LAUNCH_CHECK();
    stencil3d_fixup_kernel<T, M><<<fb, 256, 0, st>>>(a, q, main_blocks);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

long long v3_face_count(const Grid& g, int max_threads, int ctas_per_sm) {
    if (!v2_applicable(g)) return 0;
    return v2_geometry(g, std::max(1, ctas_per_sm) * kNumSMs, max_threads).face_count;
}

template <Prob P, Mode M, int MINB>
static jfnk_status launch_v3_pmb(const StencilArgs<float>& a, cudaStream_t st) {
    // z chunks for MINB resident CTAs per SM
    const V2Geom q = v2_geometry(a.g, MINB * kNumSMs, a.v2_threads);
    if ((q.n / 2) * q.BY > kV3Threads) {
        set_error("paired-element kernel: CTA of %d x %d threads", q.n / 2, q.BY);
        return JFNK_ERR_INVALID_ARG;
    }
    if (q.face_count > a.face_cap) {
        set_error("face scratch too small (%lld < %lld)", a.face_cap, q.face_count);
        return JFNK_ERR_WORKSPACE;
    }
    const int main_blocks = q.Ty * q.Tz;
    const int fb = fixup_blocks(q);
    if (main_blocks + fb > kMaxRedBlocks * 2) {
        set_error("v3 grid too large for the reduction scratch");
        return JFNK_ERR_INVALID_ARG;
    }
    const size_t NP = (size_t)q.n + 2;
    const size_t smem = sizeof(float) * (3 * (size_t)(q.BY + 1) * NP + 16 * (size_t)q.BY * NP);
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose attributes are set
    const unsigned long long dbit = device_bit();
    if (!(attr_devs.load() & dbit)) {
        JFNK_CUDA_TRY(cudaFuncSetAttribute(stencil3d_v3_kernel<P, M, MINB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024 / MINB));
        JFNK_CUDA_TRY(cudaFuncSetAttribute(stencil3d_v3_kernel<P, M, MINB>,
                                           cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        attr_devs.fetch_or(dbit);
    }
    stencil3d_v3_kernel<P, M, MINB><<<dim3(q.Ty, q.Tz), dim3(q.n / 2, q.BY), smem, st>>>(a, q);
    JFNK_LAUNCH_CHECK();
    stencil3d_fixup_kernel<float, M><<<fb, 256, 0, st>>>(a, q, main_blocks);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

// a.v3 = 1: one CTA per SM (up to 128 registers a thread); 2: two CTAs per SM
// (64 registers; the modes that read a direction spill 100-190 bytes a thread
// to local memory); otherwise (the default) two for the residual, whose loads
// are half as many and which spills 16-28 bytes, and one for the other modes:
// the faster choice for each on 129^3-257^3 grids.
template <Prob P, Mode M>
static jfnk_status launch_v3_pm(const StencilArgs<float>& a, cudaStream_t st) {
    const bool two = a.v3 == 2 || (a.v3 != 1 && M == Mode::F);
    return two ? launch_v3_pmb<P, M, 2>(a, st) : launch_v3_pmb<P, M, 1>(a, st);
}

template <Prob P>
static jfnk_status launch_v3_p(Mode mode, const StencilArgs<float>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::F: return launch_v3_pm<P, Mode::F>(a, st);
        case Mode::JV: return launch_v3_pm<P, Mode::JV>(a, st);
        case Mode::BMJ: return launch_v3_pm<P, Mode::BMJ>(a, st);
        case Mode::CHEB0: return launch_v3_pm<P, Mode::CHEB0>(a, st);
        case Mode::CHEB: return launch_v3_pm<P, Mode::CHEB>(a, st);
        case Mode::CHEBLAST: return launch_v3_pm<P, Mode::CHEBLAST>(a, st);
    }
    set_error("unknown stencil mode");
    return JFNK_ERR_INVALID_ARG;
}

jfnk_status launch_stencil_v3(Prob prob, Mode mode, const StencilArgs<float>& a, cudaStream_t st) {
    if (prob == Prob::ND3) return launch_v3_p<Prob::ND3>(mode, a, st);
    if (prob == Prob::NDK3) return launch_v3_p<Prob::NDK3>(mode, a, st);
    set_error("v3 kernel is 3D only");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T, Prob P>
static jfnk_status launch_v2_p(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::F: return launch_v2_pm<T, P, Mode::F>(a, st);
        case Mode::JV: return launch_v2_pm<T, P, Mode::JV>(a, st);
        case Mode::BMJ: return launch_v2_pm<T, P, Mode::BMJ>(a, st);
        case Mode::CHEB0: return launch_v2_pm<T, P, Mode::CHEB0>(a, st);
        case Mode::CHEB: return launch_v2_pm<T, P, Mode::CHEB>(a, st);
        case Mode::CHEBLAST: return launch_v2_pm<T, P, Mode::CHEBLAST>(a, st);
    }
    set_error("unknown stencil mode");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
jfnk_status launch_stencil_v2(Prob prob, Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    if (prob == Prob::ND3) return launch_v2_p<T, Prob::ND3>(mode, a, st);
    if (prob == Prob::NDK3) return launch_v2_p<T, Prob::NDK3>(mode, a, st);
    set_error("v2 kernel is 3D only");
    return JFNK_ERR_INVALID_ARG;
}

template jfnk_status launch_stencil_v2<double>(Prob, Mode, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_stencil_v2<float>(Prob, Mode, const StencilArgs<float>&, cudaStream_t);

}  // namespace jfnk
