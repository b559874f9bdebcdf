// Element-parallel 3D element-residual kernels.
//
// Phase 1 (elements): one thread per element gathers its 8 nodal values of
// w = x + eps v (boundary entries of v ignored), evaluates the element
// residual (or its vector-Jacobian product) and stores the 8 nodal
// contributions in a scratch array C[corner][element].  No shared memory and
// no barrier: every element of the level is independent, so all SMs stay busy
// whatever the grid size, and no element is evaluated twice.
// Phase 2 (nodes): one thread per node sums the contributions of its 8
// elements in a fixed order, applies the node factor and the fused epilogue of
// the mode, and the last block completes the norm reduction (deterministic).
//
// Each F_i is the same sum of element integrals as in the tiled kernels; the
// price is 2 x 8 scratch words per element of extra traffic, which the FP64
// kernels (bound by the FP64 pipe by two orders of magnitude) do not notice
// and which stays in L2 on the small levels.
#include <algorithm>
#include <atomic>

#include <cooperative_groups.h>

#include "element.cuh"
#include "reduce.cuh"
#include "stencil.cuh"
#include "stencil_body.cuh"
#include "stencil_ep.cuh"

namespace jfnk {

constexpr int kEpElemThreads = 128;
constexpr int kEpNodeThreads = 256;

// Element (x, y, z): blockIdx.y = y, blockIdx.z = z, x = blockIdx.x * blockDim.x
// + threadIdx.x, so a warp holds consecutive elements of one x-row.  Each
// thread forms w = x + eps v at its 4 left corners (x, y+dy, z+dz) and takes the
// 4 right corners from its neighbour lane (the left corners of element x+1);
// the last element of a row and lane 31 form theirs themselves.  32-bit node
// indices: (n+1)^3 < 2^31 for every grid the launcher accepts.
template <typename T, Prob P, Mode M, bool ADJ>
__global__ void __launch_bounds__(kEpElemThreads) ep3d_elem_kernel(const StencilArgs<T> a) {
    const int n = a.g.n;
    const int sy = (int)a.g.sy, sz = (int)a.g.sz;
    const long long ne = (long long)n * n * n;
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = x < n;
    T eps = T(0);
    if (!ADJ && M != Mode::F) eps = eps_of<T>(a.eps);
    const bool yz_in0 = y > 0, yz_in1 = y + 1 < n, z_in0 = z > 0, z_in1 = z + 1 < n;
    // node value (w, or u with the masked direction in vv for the adjoint) at (X, y+dy, z+dz)
    auto corner = [&](int X, int dy, int dz, T& wv, T& vv) {
        const int idx = (int)JFNK_IDX((z + dz) * sz + (y + dy) * sy + X, a.g.size);
        const bool bnd = X == 0 || X == n || (dy ? !yz_in1 : !yz_in0) || (dz ? !z_in1 : !z_in0);
        T uv = a.u[idx];
        vv = T(0);
        if (ADJ) {
            vv = bnd ? T(0) : a.v[idx];
        } else if (M != Mode::F) {
            if (!bnd) uv += eps * a.v[idx];
        }
        wv = uv;
    };
    const int xl = valid ? x : n - 1;  // inactive lanes still take part in the shuffles
    T wl[4], vl[4], wr[4], vr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) corner(xl, k & 1, k >> 1, wl[k], vl[k]);
    const bool own_right = (lane == 31) || (xl == n - 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        wr[k] = __shfl_down_sync(0xffffffffu, wl[k], 1);
        if (ADJ) vr[k] = __shfl_down_sync(0xffffffffu, vl[k], 1);
    }
    if (own_right) {
#pragma unroll
        for (int k = 0; k < 4; ++k) corner(xl + 1, k & 1, k >> 1, wr[k], vr[k]);
    }
    if (!valid) return;
    const long long e = ((long long)z * n + y) * n + x;
    // corner c = dx + 2 dy + 4 dz
    T ue[8] = {wl[0], wr[0], wl[1], wr[1], wl[2], wr[2], wl[3], wr[3]};
    T r[8];
    if (ADJ) {
        T ve[8] = {vl[0], vr[0], vl[1], vr[1], vl[2], vr[2], vl[3], vr[3]};
        T dk;
        elem_vjp3<T>(ue, ve, P == Prob::NDK3 ? a.kappa[e] : T(1), r, dk);
        if (a.dkout) a.dkout[e] = dk * a.dk_scale;
    } else if (P == Prob::NDK3) {
        elem_nd3<T, true>(ue, a.kappa[e], r);
    } else {
        elem_nd3<T, false>(ue, T(1), r);
    }
    T* C = a.face + JFNK_IDX(e, ne);
#pragma unroll
    for (int c = 0; c < 8; ++c) C[c * ne] = r[c];
}

// Nodes in storage order, one per thread, grid-strided over the blocks (the
// last-block reduction holds at most 2 kMaxRedBlocks partials): every thread
// of every block has a node on all levels, including rows of n+1 nodes that
// do not fill whole blocks.
template <typename T, Mode M, bool ADJ>
__global__ void __launch_bounds__(kEpNodeThreads) ep3d_node_kernel(const StencilArgs<T> a) {
    __shared__ double red_sm[32];
    const Grid g = a.g;
    const int n = g.n, NP = n + 1;
    const long long ne = (long long)n * n * n;
    const int esy = n, esz = n * n;  // element strides
    const int nodes = NP * NP * NP;  // node index = Z sz + Y sy + X (dense grid)
    const T* C = a.face;
    T inv_eps = T(0);
    if (!ADJ && M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    const T ns = a.node_scale, ns_inv = a.node_scale * inv_eps;
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nodes; idx += gridDim.x * blockDim.x) {
        const int X = idx % NP, YZ = idx / NP;
        const int Y = YZ % NP, Z = YZ / NP;
        const bool inner = X > 0 && X < n && Y > 0 && Y < n && Z > 0 && Z < n;
        T sum = T(0);
        if (inner) {
            // element with corner c = dx + 2 dy + 4 dz at this node: (X-dx, Y-dy, Z-dz)
            const T* Cn = C + JFNK_IDX(Z * esz + Y * esy + X - esz - esy - 1, ne - esz - esy - 1) + esz + esy + 1;
            const T c0 = Cn[0], c1 = Cn[ne - 1];
            const T c2 = Cn[2 * ne - esy], c3 = Cn[3 * ne - esy - 1];
            const T c4 = Cn[4 * ne - esz], c5 = Cn[5 * ne - esz - 1];
            const T c6 = Cn[6 * ne - esz - esy], c7 = Cn[7 * ne - esz - esy - 1];
            sum = ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7));
        }
        if (ADJ)
            epilogue_adj<T, M>(a, idx, inner, sum * ns, ck, red);
        else
            epilogue<T, M, true>(a, idx, inner, sum, inv_eps, ck, red, ns, ns_inv);
    }
    stencil_reduce(a, red, red_sm);
}

// ---------------------------------------------------------------------------
// z-marching element columns.  Thread (x, y) evaluates the elements
// (x, y, z) for z in its chunk, in order.  Neighbouring elements of a column
// share a z face: the x/y butterflies of the face's nodal values
// (elem_nd3_mid's a/b inputs) are computed once per face instead of once per
// element, and on the test-function side the two elements' face modes are
// summed before the y and x passes, so each face's 4 node sums leave the
// thread already added over z.  The column's 4 per-plane node values go to
// scratch Cz[k][z][y][x] (k = a + 2b: node (x+a, y+b, z)); the node kernel
// adds the 4 columns around each node.  Against one element per thread this
// saves 19 of ~183 operations per node (forward face butterflies, half the
// nodal w = x + eps v, the y/x passes of one face, 4 of the 7 node adds) and
// half of the scratch traffic.  A chunk that starts at z0 > 0 evaluates element
// z0 - 1 once more (only its upper face modes are kept), so every interior
// plane is completed inside one chunk and written once.
// Selected per precision by zm_min_n (off by default: measured against one
// element a thread it ran 5-20 % slower in FP64 and within +-10 % of the
// halo-free kernel in FP32; a variant that also added x neighbours through
// warp shuffles, halving the scratch again, was slower still).
// ---------------------------------------------------------------------------
constexpr int kZmThreads = 128;

template <typename T, Prob P, Mode M>
__global__ void __launch_bounds__(kZmThreads) zm3d_elem_kernel(const StencilArgs<T> a, int zchunk) {
    const int n = a.g.n;
    const int sy = (int)a.g.sy, sz = (int)a.g.sz;
    const int y = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = x < n;
    const int xl = valid ? x : n - 1;  // inactive lanes still take part in the shuffles
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(n, z0 + zchunk);
    const int zs = z0 > 0 ? z0 - 1 : 0;
    T eps = T(0);
    if (M != Mode::F) eps = eps_of<T>(a.eps);
    const bool y_in0 = y > 0, y_in1 = y + 1 < n;
    const bool own_right = (lane == 31) || (xl == n - 1);
    // raw u (and v) of node (X, y + dy, Z); w = u + eps v formed by `wval`
    auto load = [&](int X, int dy, int Z, T& uv, T& vv) {
        const int idx = (int)JFNK_IDX(Z * sz + (y + dy) * sy + X, a.g.size);
        uv = a.u[idx];
        vv = T(0);
        if (M != Mode::F) {
            const bool bnd = X == 0 || X == n || (dy ? !y_in1 : !y_in0) || Z == 0 || Z == n;
            if (!bnd) vv = a.v[idx];
        }
    };
    // this thread's loads of plane Z: left nodes of rows y, y+1, and the right
    // ones where no neighbour lane holds them
    struct Raw {
        T u0, v0, u1, v1, ur0, vr0, ur1, vr1;
    };
    auto fetch = [&](int Z, Raw& r) {
        load(xl, 0, Z, r.u0, r.v0);
        load(xl, 1, Z, r.u1, r.v1);
        if (own_right) {
            load(xl + 1, 0, Z, r.ur0, r.vr0);
            load(xl + 1, 1, Z, r.ur1, r.vr1);
        }
    };
    // face butterflies of a plane: s0 = p_0 + p_1, s1 = p_1 - p_0, s2 = q_0 + q_1,
    // s3 = q_1 - q_0 with p_b / q_b the x sum / difference of row y + b
    auto face = [&](const Raw& r, T& s0, T& s1, T& s2, T& s3) {
        T l0 = r.u0, l1 = r.u1;
        if (M != Mode::F) {
            l0 = l0 + eps * r.v0;
            l1 = l1 + eps * r.v1;
        }
        T r0 = __shfl_down_sync(0xffffffffu, l0, 1);
        T r1 = __shfl_down_sync(0xffffffffu, l1, 1);
        if (own_right) {
            r0 = r.ur0;
            r1 = r.ur1;
            if (M != Mode::F) {
                r0 = r0 + eps * r.vr0;
                r1 = r1 + eps * r.vr1;
            }
        }
        const T p0 = l0 + r0, q0 = r0 - l0;
        const T p1 = l1 + r1, q1 = r1 - l1;
        s0 = p0 + p1;
        s1 = p1 - p0;
        s2 = q0 + q1;
        s3 = q1 - q0;
    };
    const long long ks = zm3d_plane_stride(n);
    T* Cz = a.face;
    const int col = y * n + x;
    Raw cur;
    fetch(zs, cur);
    T a00, a01, a10, a11;
    face(cur, a00, a01, a10, a11);
    fetch(zs + 1, cur);
    Raw nxt = cur;
    T k00 = T(0), k01 = T(0), k10 = T(0), k11 = T(0);  // upper-face modes of the element below
    T kap = T(1), kap_n = T(1);
    if (P == Prob::NDK3 && valid) kap = a.kappa[JFNK_IDX((zs * n + y) * n + x, (long long)n * n * n)];
    for (int z = zs; z < z1; ++z) {
        // prefetch the plane above the next element
        if (z + 2 <= n) fetch(z + 2, nxt);
        if (P == Prob::NDK3 && valid && z + 1 < z1) kap_n = a.kappa[JFNK_IDX(((z + 1) * n + y) * n + x, (long long)n * n * n)];
        T b00, b01, b10, b11;
        face(cur, b00, b01, b10, b11);
        T R001, R010, R011, R100, R101, R110, R111;
        elem_nd3_mid<T, P == Prob::NDK3>(a00, a01, a10, a11, b00, b01, b10, b11, kap, R001, R010, R011, R100,
                                         R101, R110, R111);
        // z pass: lower-face (c = 0) and upper-face (c = 1) modes
        const T e01_0 = R010 - R011, e01_1 = R010 + R011;
        const T e10_0 = R100 - R101, e10_1 = R100 + R101;
        const T e11_0 = R110 - R111, e11_1 = R110 + R111;
        if (valid && z >= z0 && z >= 1) {
            // plane z: this element's lower face plus the element below's upper face
            const T E00 = k00 - R001, E01 = k01 + e01_0, E10 = k10 + e10_0, E11 = k11 + e11_0;
            const T f0_0 = E00 - E01, f0_1 = E00 + E01;  // y pass, p = 0, b = 0 / 1
            const T f1_0 = E10 - E11, f1_1 = E10 + E11;  // p = 1
            T* Cp = Cz + JFNK_IDX((long long)z * n * n + col, ks);
            Cp[0] = f0_0 - f1_0;       // node (x,   y,   z)
            Cp[ks] = f0_0 + f1_0;      // node (x+1, y,   z)
            Cp[2 * ks] = f0_1 - f1_1;  // node (x,   y+1, z)
            Cp[3 * ks] = f0_1 + f1_1;  // node (x+1, y+1, z)
        }
        k00 = R001;
        k01 = e01_1;
        k10 = e10_1;
        k11 = e11_1;
        a00 = b00;
        a01 = b01;
        a10 = b10;
        a11 = b11;
        cur = nxt;
        kap = kap_n;
    }
}

// Node phase of the z-marching kernel: the 4 columns around node (X, Y, Z),
// in a fixed order, then the epilogue of the mode and the norm reduction.
template <typename T, Mode M>
__global__ void __launch_bounds__(kEpNodeThreads) zm3d_node_kernel(const StencilArgs<T> a) {
    __shared__ double red_sm[32];
    const int n = a.g.n, NP = n + 1;
    const int nodes = NP * NP * NP;
    const long long ks = zm3d_plane_stride(n);
    const T* Cz = a.face;
    T inv_eps = T(0);
    if (M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nodes; idx += gridDim.x * blockDim.x) {
        const int X = idx % NP, YZ = idx / NP;
        const int Y = YZ % NP, Z = YZ / NP;
        const bool inner = X > 0 && X < n && Y > 0 && Y < n && Z > 0 && Z < n;
        T val = T(0);
        if (inner) {
            const T* Cp = Cz + JFNK_IDX((long long)Z * n * n + (Y - 1) * n + X - 1, ks - n - 1) + n + 1;
            const T c0 = Cp[0], c1 = Cp[ks - 1];
            const T c2 = Cp[2 * ks - n], c3 = Cp[3 * ks - n - 1];
            val = ((c0 + c1) + (c2 + c3)) * a.node_scale;
        }
        epilogue<T, M>(a, idx, inner, val, inv_eps, ck, red);
    }
    stencil_reduce(a, red, red_sm);
}

// FP32 levels with at most kEpSmallElems elements (n <= 8): both phases in one
// CTA, the contributions exchanged through shared memory and the norm reduced
// inside the block -- one launch and no grid-wide completion for the latency-
// bound small levels.  Each element takes its 8 corners itself; the element
// values and the per-node sums (same order) are those of the two kernels
// above.  (In FP64 one SM would do all the element arithmetic on its two
// FP64 lanes, which is slower than spreading it over the GPU.)
constexpr int kEpSmallThreads = 512;
constexpr int kEpSmallElems = 512;

template <typename T, Prob P, Mode M, bool ADJ>
__global__ void __launch_bounds__(kEpSmallThreads) ep3d_small_kernel(const StencilArgs<T> a) {
    __shared__ T Cs[8 * kEpSmallElems];
    __shared__ double red_sm[32];
    const int n = a.g.n, NP = n + 1;
    const int ne = n * n * n;
    const int sy = (int)a.g.sy, sz = (int)a.g.sz;
    T eps = T(0);
    if (!ADJ && M != Mode::F) eps = eps_of<T>(a.eps);
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int x = e % n, y = (e / n) % n, z = e / (n * n);
        T ue[8], ve[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int X = x + (c & 1), Y = y + ((c >> 1) & 1), Z = z + (c >> 2);
            const int idx = Z * sz + Y * sy + X;
            const bool bnd = X == 0 || X == n || Y == 0 || Y == n || Z == 0 || Z == n;
            T uv = a.u[idx];
            ve[c] = T(0);
            if (ADJ) {
                ve[c] = bnd ? T(0) : a.v[idx];
            } else if (M != Mode::F) {
                if (!bnd) uv += eps * a.v[idx];
            }
            ue[c] = uv;
        }
        T r[8];
        if (ADJ) {
            T dk;
            elem_vjp3<T>(ue, ve, P == Prob::NDK3 ? a.kappa[e] : T(1), r, dk);
            if (a.dkout) a.dkout[e] = dk * a.dk_scale;
        } else if (P == Prob::NDK3) {
            elem_nd3<T, true>(ue, a.kappa[e], r);
        } else {
            elem_nd3<T, false>(ue, T(1), r);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) Cs[c * ne + e] = r[c];
    }
    __syncthreads();
    T inv_eps = T(0);
    if (!ADJ && M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    const int esy = n, esz = n * n;
    float red = 0.f;
    for (int idx = threadIdx.x; idx < NP * NP * NP; idx += blockDim.x) {
        const int X = idx % NP, YZ = idx / NP;
        const int Y = YZ % NP, Z = YZ / NP;
        const bool inner = X > 0 && X < n && Y > 0 && Y < n && Z > 0 && Z < n;
        T val = T(0);
        if (inner) {
            const T* Cn = Cs + (Z * esz + Y * esy + X);
            const T c0 = Cn[0], c1 = Cn[ne - 1];
            const T c2 = Cn[2 * ne - esy], c3 = Cn[3 * ne - esy - 1];
            const T c4 = Cn[4 * ne - esz], c5 = Cn[5 * ne - esz - 1];
            const T c6 = Cn[6 * ne - esz - esy], c7 = Cn[7 * ne - esz - esy - 1];
            val = (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7))) * a.node_scale;
        }
        if (ADJ)
            epilogue_adj<T, M>(a, idx, inner, val, ck, red);
        else
            epilogue<T, M>(a, idx, inner, val, inv_eps, ck, red);
    }
    if (a.red == RedOut::NONE) return;
    const double bs = block_sum(red, red_sm);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(bs);
        if (a.red_norm) *a.red_norm = nrm;
        if (a.red == RedOut::EPS || a.red == RedOut::EPS_UNIT)
            set_eps_slot(a.red_eps, a.epsp, nrm, a.red == RedOut::EPS_UNIT, a.status);
    }
}

// FP32 levels with n <= kEpClusterMaxN: the level in one thread-block
// cluster of up to 16 CTAs, the contributions in distributed shared memory.
// CTA r of the cluster owns element slices z in [r S, r S + S) (S = ceil(n /
// 16)) and the node planes with the same z (the last CTA also plane n).  A
// node plane takes its lower-z elements' contributions from the CTA below
// through DSMEM after a cluster barrier; the norm is summed over the CTAs' block
// sums in rank order.  One launch and no round trip through global memory or a
// completion counter, for levels whose two-launch form is a chain of
// latencies.  The element values and the per-node sums (same order) are those
// of the element-parallel pair.
constexpr int kEpClusterThreads = 1024;
constexpr int kEpClusterMaxCtas = 16;
constexpr int kEpClusterMaxN = 32;  // S <= 2: 8 S n^2 words = 64 KB of shared memory at n = 32

__host__ __device__ inline int ep3d_cluster_slices(int n) { return (n + kEpClusterMaxCtas - 1) / kEpClusterMaxCtas; }
__host__ __device__ inline int ep3d_cluster_ctas(int n) {
    const int S = ep3d_cluster_slices(n);
    return (n + S - 1) / S;
}

template <typename T, Prob P, Mode M>
__global__ void __launch_bounds__(kEpClusterThreads) ep3d_cluster_kernel(const StencilArgs<T> a) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Cs = reinterpret_cast<T*>(smem_raw);  // [8][S][n][n]: this CTA's element contributions
    __shared__ double red_sm[32];
    __shared__ double bsums[kEpClusterMaxCtas];  // rank 0: every CTA's block sum
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    const int n = a.g.n, NP = n + 1, nn = n * n;
    const int S = ep3d_cluster_slices(n);
    const int E = S * nn;  // stride of a corner in every CTA's array
    const int z0 = rank * S;
    const int z1 = min(z0 + S, n);
    const int sy = (int)a.g.sy, sz = (int)a.g.sz;
    T eps = T(0);
    if (M != Mode::F) eps = eps_of<T>(a.eps);
    for (int e = threadIdx.x; e < (z1 - z0) * nn; e += blockDim.x) {
        const int x = e % n, y = (e / n) % n, z = z0 + e / nn;
        T ue[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int X = x + (c & 1), Y = y + ((c >> 1) & 1), Z = z + (c >> 2);
            const int idx = (int)JFNK_IDX(Z * sz + Y * sy + X, a.g.size);
            const bool bnd = X == 0 || X == n || Y == 0 || Y == n || Z == 0 || Z == n;
            T uv = a.u[idx];
            if (M != Mode::F && !bnd) uv += eps * a.v[idx];
            ue[c] = uv;
        }
        T r[8];
        if (P == Prob::NDK3)
            elem_nd3<T, true>(ue, a.kappa[JFNK_IDX(z * nn + y * n + x, (long long)nn * n)], r);
        else
            elem_nd3<T, false>(ue, T(1), r);
#pragma unroll
        for (int c = 0; c < 8; ++c) Cs[c * E + e] = r[c];
    }
    cluster.sync();
    // the CTA below holds slice z0 - 1, its last (S is full for every CTA but the last)
    const T* Cd = rank > 0 ? cluster.map_shared_rank(Cs, rank - 1) : Cs;
    T inv_eps = T(0);
    if (M != Mode::F) inv_eps = inv_eps_of<T>(a.eps);
    ChebK<T> ck = {T(0), T(0), T(0)};
    if (M == Mode::CHEB0 || M == Mode::CHEB || M == Mode::CHEBLAST) ck = cheb_of<T>(a.cheb, a.cheb_step);
    float red = 0.f;
    const int zend = (rank == ncta - 1) ? NP : z1;
    for (int i = threadIdx.x; i < (zend - z0) * NP * NP; i += blockDim.x) {
        const int X = i % NP, YZ = i / NP;
        const int Y = YZ % NP, Z = z0 + YZ / NP;
        const bool inner = X > 0 && X < n && Y > 0 && Y < n && Z > 0 && Z < n;
        T val = T(0);
        if (inner) {
            // corner c of element (X - dx, Y - dy, Z - dz), c = dx + 2 dy + 4 dz
            const int e0 = (int)JFNK_IDX((Z - z0) * nn + Y * n + X, E);  // element (X, Y, Z), this CTA
            const T c0 = Cs[e0], c1 = Cs[E + e0 - 1];
            const T c2 = Cs[2 * E + e0 - n], c3 = Cs[3 * E + e0 - n - 1];
            const T* Cl = (Z > z0) ? Cs : Cd;                            // slice Z - 1
            const int e1 = (int)JFNK_IDX(((Z > z0) ? (Z - 1 - z0) : (S - 1)) * nn + Y * n + X, E);
            const T c4 = Cl[4 * E + e1], c5 = Cl[5 * E + e1 - 1];
            const T c6 = Cl[6 * E + e1 - n], c7 = Cl[7 * E + e1 - n - 1];
            val = (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7))) * a.node_scale;
        }
        epilogue<T, M>(a, (int)JFNK_IDX(Z * sz + Y * sy + X, a.g.size), inner, val, inv_eps, ck, red);
    }
    if (a.red != RedOut::NONE) {
        const double bs = block_sum(red, red_sm);
        if (threadIdx.x == 0) *cluster.map_shared_rank(&bsums[rank], 0) = bs;
    }
    // every CTA is done with its neighbour's contributions and has posted its
    // block sum to rank 0; after this barrier no CTA touches another's memory
    cluster.sync();
    if (a.red != RedOut::NONE && rank == 0 && threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < ncta; ++q) tot += bsums[q];
        const double nrm = sqrt(tot);
        if (a.red_norm) *a.red_norm = nrm;
        if (a.red == RedOut::EPS || a.red == RedOut::EPS_UNIT)
            set_eps_slot(a.red_eps, a.epsp, nrm, a.red == RedOut::EPS_UNIT, a.status);
    }
}

template <Prob P, Mode M>
static cudaError_t ep3d_cluster_attrs() {
    auto k = ep3d_cluster_kernel<float, P, M>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(8 * 2 * kEpClusterMaxN * kEpClusterMaxN * sizeof(float)));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <Prob P>
static cudaError_t ep3d_cluster_attrs_p() {
    cudaError_t e = ep3d_cluster_attrs<P, Mode::F>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs<P, Mode::JV>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs<P, Mode::BMJ>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs<P, Mode::CHEB0>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs<P, Mode::CHEB>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs<P, Mode::CHEBLAST>();
    return e;
}

bool ep3d_cluster_init() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    static std::atomic<int> ok[64];  // per device: 0 unknown, 1 usable, -1 not
    if (dev < 0 || dev >= 64) return false;
    if (ok[dev].load() != 0) return ok[dev].load() > 0;
    cudaError_t e = ep3d_cluster_attrs_p<Prob::ND3>();
    if (e == cudaSuccess) e = ep3d_cluster_attrs_p<Prob::NDK3>();
    int clusters = 0;
    if (e == cudaSuccess) {
        // the largest launch (n = kEpClusterMaxN) must fit on the device
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ep3d_cluster_ctas(kEpClusterMaxN);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(ep3d_cluster_ctas(kEpClusterMaxN));
        cfg.blockDim = dim3(kEpClusterThreads);
        cfg.dynamicSmemBytes = 8 * 2 * kEpClusterMaxN * kEpClusterMaxN * sizeof(float);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&clusters, ep3d_cluster_kernel<float, Prob::ND3, Mode::CHEB>, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();  // clear: the pair of kernels runs instead
    ok[dev].store((e == cudaSuccess && clusters > 0) ? 1 : -1);
    return ok[dev].load() > 0;
}

template <typename T, Prob P, Mode M>
static jfnk_status launch_ep3d_cluster(const StencilArgs<T>& a, cudaStream_t st) {
    const int n = a.g.n;
    const int ncta = ep3d_cluster_ctas(n);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(kEpClusterThreads);
    cfg.dynamicSmemBytes = 8ull * ep3d_cluster_slices(n) * n * n * sizeof(T);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, ep3d_cluster_kernel<T, P, M>, a);
    if (e != cudaSuccess) {
        set_error("cluster launch: %s", cudaGetErrorString(e));
        return JFNK_ERR_CUDA;
    }
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, Prob P, Mode M, bool ADJ>
static jfnk_status launch_ep3d_pm(const StencilArgs<T>& a, cudaStream_t st) {
    const Grid& g = a.g;
    const bool zm = !ADJ && a.zm_min_n > 0 && g.n >= a.zm_min_n;
    if (ep3d_scratch_need(g, zm) > a.face_cap) {
        set_error("element scratch too small (%lld < %lld)", a.face_cap, ep3d_scratch_need(g, zm));
        return JFNK_ERR_WORKSPACE;
    }
    if (g.n > 1024) {
        set_error("element-parallel kernels: n = %d beyond 1024 (32-bit node indices, grid rows)", g.n);
        return JFNK_ERR_INVALID_ARG;
    }
    if constexpr (sizeof(T) == 4 && !ADJ) {
        if (g.n >= a.cl_min_n && g.n <= std::min(a.cl_max_n, kEpClusterMaxN) && ep3d_cluster_init())
            return launch_ep3d_cluster<T, P, M>(a, st);
    }
    if (sizeof(T) == 4 && (long long)g.n * g.n * g.n <= kEpSmallElems) {
        ep3d_small_kernel<T, P, M, ADJ><<<1, kEpSmallThreads, 0, st>>>(a);
        JFNK_LAUNCH_CHECK();
        return JFNK_OK;
    }
    // x-rows of up to 128 elements per block (a whole number of warps)
    const int bx = std::min(kEpElemThreads, ((g.n + 31) / 32) * 32);
    if (zm) {
        // z chunks so that enough threads march at once: about 39k (8 warps
        // per SM) in FP64, whose element arithmetic alone keeps the FP64 pipe
        // busy, and 156k (32 warps per SM) in FP32, where the loads of the next
        // plane have to be hidden behind other warps' arithmetic
        const long long cols = (long long)g.n * g.n;
        const long long target = sizeof(T) == 8 ? 38912 : 155648;
        const int chunks = (int)std::max<long long>(1, std::min<long long>(g.n, (target + cols - 1) / cols));
        const int zchunk = (g.n + chunks - 1) / chunks;
        const int nzc = (g.n + zchunk - 1) / zchunk;
        zm3d_elem_kernel<T, P, M><<<dim3((g.n + bx - 1) / bx, g.n, nzc), bx, 0, st>>>(a, zchunk);
        JFNK_LAUNCH_CHECK();
        const long long nodes = (long long)(g.n + 1) * (g.n + 1) * (g.n + 1);
        const int nb = (int)std::min<long long>((nodes + kEpNodeThreads - 1) / kEpNodeThreads, 2LL * kMaxRedBlocks);
        zm3d_node_kernel<T, M><<<nb, kEpNodeThreads, 0, st>>>(a);
        JFNK_LAUNCH_CHECK();
        return JFNK_OK;
    }
    ep3d_elem_kernel<T, P, M, ADJ><<<dim3((g.n + bx - 1) / bx, g.n, g.n), bx, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    // the reduction scratch holds 2 kMaxRedBlocks partials: nodes grid-strided beyond
    const long long nodes = (long long)(g.n + 1) * (g.n + 1) * (g.n + 1);
    const int nb = (int)std::min<long long>((nodes + kEpNodeThreads - 1) / kEpNodeThreads, 2LL * kMaxRedBlocks);
    ep3d_node_kernel<T, M, ADJ><<<nb, kEpNodeThreads, 0, st>>>(a);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

template <typename T, Prob P, bool ADJ>
static jfnk_status launch_ep3d_p(Mode mode, const StencilArgs<T>& a, cudaStream_t st) {
    switch (mode) {
        case Mode::F:
            if constexpr (!ADJ) return launch_ep3d_pm<T, P, Mode::F, false>(a, st);
            break;
        case Mode::JV: return launch_ep3d_pm<T, P, Mode::JV, ADJ>(a, st);
        case Mode::BMJ: return launch_ep3d_pm<T, P, Mode::BMJ, ADJ>(a, st);
        case Mode::CHEB0: return launch_ep3d_pm<T, P, Mode::CHEB0, ADJ>(a, st);
        case Mode::CHEB: return launch_ep3d_pm<T, P, Mode::CHEB, ADJ>(a, st);
        case Mode::CHEBLAST: return launch_ep3d_pm<T, P, Mode::CHEBLAST, ADJ>(a, st);
    }
    set_error("mode not available for the element-parallel kernels");
    return JFNK_ERR_INVALID_ARG;
}

template <typename T>
jfnk_status launch_ep3d(Prob prob, Mode mode, bool adj, const StencilArgs<T>& a, cudaStream_t st) {
    if (prob == Prob::ND3)
        return adj ? launch_ep3d_p<T, Prob::ND3, true>(mode, a, st) : launch_ep3d_p<T, Prob::ND3, false>(mode, a, st);
    if (prob == Prob::NDK3)
        return adj ? launch_ep3d_p<T, Prob::NDK3, true>(mode, a, st)
                   : launch_ep3d_p<T, Prob::NDK3, false>(mode, a, st);
    set_error("the element-parallel kernels are 3D only");
    return JFNK_ERR_INVALID_ARG;
}

template jfnk_status launch_ep3d<double>(Prob, Mode, bool, const StencilArgs<double>&, cudaStream_t);
template jfnk_status launch_ep3d<float>(Prob, Mode, bool, const StencilArgs<float>&, cudaStream_t);

}  // namespace jfnk
