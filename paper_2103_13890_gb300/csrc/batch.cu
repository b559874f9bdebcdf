// Batched kernels: one launch applies a level operation to all active
// instances of a batch (see batch.cuh).  The per-instance work is exactly the
// single-problem kernels' work (the 2D row-segment body and the vector
// operations are the same code paths); only the mapping of CTAs to
// (instance, tile/block) comes from a work list, and reductions complete per
// instance.
#include "batch.cuh"
#include "reduce.cuh"
#include "stencil_body.cuh"

namespace jfnk {

constexpr int kBThreads = 256;

// ---------------------------------------------------------------------------
// 2D element-residual kernel over (instance, row segment, row chunk) tiles
// ---------------------------------------------------------------------------
// Persistent over the work list: CTA b processes tiles b, b + gridDim.x, ...
// (gridDim.x = ntiles gives one tile per CTA).
template <typename T, Mode M>
__global__ void __launch_bounds__(512) stencil2d_batched_kernel(const StencilArgs<T>* __restrict__ args,
                                                                 const BTile* __restrict__ tiles, int ntiles) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ double red_sm[32];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const BTile t = tiles[k];
        stencil2d_body<T, M>(args[t.inst], t.x0, t.y0, t.y1, t.txo, t.bid, t.nblk, smem_raw, red_sm);
        __syncthreads();  // shared rows are reused by the next tile
    }
}

template <typename T>
jfnk_status launch_stencil2d_batched(Mode mode, const StencilArgs<T>* dev_args, const BTile* dev_tiles, int ntiles,
                                     int bx, cudaStream_t st, int grid) {
    if (ntiles <= 0) return JFNK_OK;
    const int g = (grid > 0 && grid < ntiles) ? grid : ntiles;
    const size_t smem = sizeof(T) * (2 * (bx + 1) + 4 * bx);
#define JFNK_B2(MM) stencil2d_batched_kernel<T, MM><<<g, bx, smem, st>>>(dev_args, dev_tiles, ntiles)
    switch (mode) {
        case Mode::F: JFNK_B2(Mode::F); break;
        case Mode::JV: JFNK_B2(Mode::JV); break;
        case Mode::BMJ: JFNK_B2(Mode::BMJ); break;
        case Mode::CHEB0: JFNK_B2(Mode::CHEB0); break;
        case Mode::CHEB: JFNK_B2(Mode::CHEB); break;
        case Mode::CHEBLAST: JFNK_B2(Mode::CHEBLAST); break;
    }
#undef JFNK_B2
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status launch_stencil2d_batched<double>(Mode, const StencilArgs<double>*, const BTile*, int, int,
                                                      cudaStream_t, int);
template jfnk_status launch_stencil2d_batched<float>(Mode, const StencilArgs<float>*, const BTile*, int, int,
                                                     cudaStream_t, int);

// ---------------------------------------------------------------------------
// batched vector operations
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool b_inner(const Grid& g, long long i) { return grid_unknown(g, i); }

__device__ __forceinline__ void b_finish_eps(const BVec& d, double nrm) {
    if (!d.slot) return;
    double e = eps_formula(d.ep.mode, d.ep.n_unknowns, *d.ep.xstat, nrm);
    double inv = e > 0.0 ? 1.0 / e : 0.0;
    d.slot->e = e;
    d.slot->inv = inv;
    d.slot->ef = (float)e;
    d.slot->invf = (float)inv;
}

__device__ __forceinline__ uint64_t b_splitmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T, BOp OP>
__global__ void __launch_bounds__(kBThreads) bvec_kernel(const BVec* __restrict__ descs, const BItem* __restrict__ items) {
    __shared__ double sm[32];
    const BItem it = items[blockIdx.x];
    const BVec& d = descs[it.inst];
    const long long stride = (long long)it.nblk * blockDim.x;
    const long long i0 = (long long)it.bid * blockDim.x + threadIdx.x;
    if (OP == BOp::CAST_D2T) {
        for (long long i = i0; i < d.g.size; i += stride) ((T*)d.y)[i] = (T)((const double*)d.x)[i];
    } else if (OP == BOp::CAST_T2D) {
        for (long long i = i0; i < d.g.size; i += stride) ((double*)d.y)[i] = (double)((const T*)d.x)[i];
    } else if (OP == BOp::COPY_T) {
        for (long long i = i0; i < d.g.size; i += stride) ((T*)d.y)[i] = ((const T*)d.x)[i];
    } else if (OP == BOp::AXPBY_D) {
        for (long long i = i0; i < d.g.size; i += stride)
            ((double*)d.y)[i] = d.a * ((const double*)d.x)[i] + d.b * ((double*)d.y)[i];
    } else if (OP == BOp::ADDSC_D) {
        for (long long i = i0; i < d.g.size; i += stride)
            ((double*)d.y)[i] = ((const double*)d.x)[i] + d.a * ((const double*)d.x2)[i];
    } else if (OP == BOp::CAST_SCALE_INT_D) {
        for (long long i = i0; i < d.g.size; i += stride)
            ((double*)d.y)[i] = b_inner(d.g, i) ? d.a * ((const double*)d.x)[i] : 0.0;
    } else if (OP == BOp::SCALE_INV_T) {
        const double nv = *d.dsc;
        const T s = (T)(nv > 0.0 ? 1.0 / nv : 0.0);
        for (long long i = i0; i < d.g.size; i += stride) ((T*)d.y)[i] = ((const T*)d.x)[i] * s;
    } else if (OP == BOp::SPLITMIX) {
        for (long long i = i0; i < d.g.size; i += stride) {
            T v = T(0);
            if (b_inner(d.g, i)) {
                const uint64_t z = b_splitmix(d.key + ((uint64_t)i + 1ULL) * 0x9E3779B97F4A7C15ULL);
                v = (T)((double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0);
            }
            ((T*)d.y)[i] = v;
        }
    } else if (OP == BOp::STAT || OP == BOp::CHEB_START) {
        double acc = 0.0;
        const double ti = (OP == BOp::CHEB_START) ? d.cheb->theta_inv : 0.0;
        for (long long i = i0; i < d.g.size; i += stride) {
            const bool in = b_inner(d.g, i);
            if (OP == BOp::STAT) {
                if (!in) continue;
                const double v = (double)((const T*)d.x)[i];
                acc += d.what == 0 ? fabs(v) : v * v;
            } else {
                const T bv = in ? ((const T*)d.x)[i] : T(0);
                const T dv = (T)((double)bv * ti);
                ((T*)d.y)[i] = bv;        // r
                ((T*)d.y2)[i] = dv;       // d
                ((T*)d.x2)[i] = T(0);     // s (written through x2's address)
                acc += (double)dv * (double)dv;
            }
        }
        const double bs = block_sum(acc, sm);
        double tot = 0.0;
        if (grid_sum_last_seg(bs, d.partials, d.counter, &tot, sm, it.bid, it.nblk) && threadIdx.x == 0) {
            const double r = (OP == BOp::STAT && d.what == 0) ? tot : sqrt(tot);
            if (d.out) *d.out = r;
            b_finish_eps(d, r);
        }
    } else if (OP == BOp::RESTRICT) {
        const Grid gc = d.gc, gf = d.g;
        const T scale = (T)d.a;
        for (long long i = i0; i < gc.size; i += stride) {
            int x, y, z;
            grid_coords(gc, i, x, y, z);
            const bool bnd = x == 0 || x == gc.nx - 1 || y == 0 || y == gc.ny - 1 ||
                             (gc.d == 3 && (z == 0 || z == gc.nz - 1));
            const long long fc = (gc.d == 3 ? (long long)(2 * z) * gf.sz : 0) + (long long)(2 * y) * gf.sy + 2 * x;
            const T* f = (const T*)d.x;
            if (bnd) {
                ((T*)d.y)[i] = d.what ? f[fc] : T(0);
                continue;
            }
            T acc = T(0);
            for (int oy = -1; oy <= 1; ++oy) {
                const T row = T(0.5) * (f[fc + oy * gf.sy - 1] + f[fc + oy * gf.sy + 1]) + f[fc + oy * gf.sy];
                acc += (oy == 0 ? T(1) : T(0.5)) * row;
            }
            ((T*)d.y)[i] = scale * acc;
        }
    } else if (OP == BOp::PROLONG_ADD) {
        const Grid gc = d.gc, gf = d.g;
        const T* c = (const T*)d.x;
        for (long long i = i0; i < gf.size; i += stride) {
            int x, y, z;
            grid_coords(gf, i, x, y, z);
            if (x == 0 || x == gf.nx - 1 || y == 0 || y == gf.ny - 1) continue;
            const int ix0 = x >> 1, ix1 = (x & 1) ? (x >> 1) + 1 : ix0;
            const int iy0 = y >> 1, iy1 = (y & 1) ? (y >> 1) + 1 : iy0;
            const T wx = (x & 1) ? T(0.5) : T(1), wy = (y & 1) ? T(0.5) : T(1);
            auto cv = [&](int cx, int cy) -> T {
                return (cx == 0 || cx == gc.nx - 1 || cy == 0 || cy == gc.ny - 1) ? T(0) : c[(long long)cy * gc.sy + cx];
            };
            T acc = wy * wx * cv(ix0, iy0);
            if (x & 1) acc += wy * wx * cv(ix1, iy0);
            if (y & 1) {
                acc += wy * wx * cv(ix0, iy1);
                if (x & 1) acc += wy * wx * cv(ix1, iy1);
            }
            ((T*)d.y)[i] += acc;
        }
    } else if (OP == BOp::MDOT) {
        // out[k] = <x, x2 + k ld>, k < m, m <= 64; each CTA reduces its share
        const double* w = (const double*)d.x;
        const double* V = (const double*)d.x2;
        for (int k0 = 0; k0 < d.m; k0 += 8) {
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.0;
            for (long long i = i0; i < d.g.size; i += stride) {
                const double wi = w[i];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (k0 + q < d.m) acc[q] += wi * V[(long long)(k0 + q) * d.ld + i];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const double bs = block_sum(acc[q], sm);
                if (threadIdx.x == 0 && k0 + q < d.m) d.partials[(long long)(k0 + q) * it.nblk + it.bid] = bs;
            }
        }
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned int prev = atomicAdd(d.counter, 1u);
            s_last = (prev == (unsigned)it.nblk - 1) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            for (int k = wid; k < d.m; k += blockDim.x >> 5) {
                double s = 0.0;
                for (int b = lane; b < it.nblk; b += 32) s += __ldcg(&d.partials[(long long)k * it.nblk + b]);
                s = warp_sum(s);
                if (lane == 0) d.out[k] = s;
            }
            if (threadIdx.x == 0) *d.counter = 0u;
        }
    } else if (OP == BOp::MAXPY_SUB) {
        double* w = (double*)d.y;
        const double* V = (const double*)d.x2;
        for (long long i = i0; i < d.g.size; i += stride) {
            double acc = w[i];
            for (int k = 0; k < d.m; ++k) acc -= d.out[k] * V[(long long)k * d.ld + i];
            w[i] = acc;
        }
    } else if (OP == BOp::COMBINE_T) {
        double* xo = (double*)d.y;
        const T* Z = (const T*)d.x;
        for (long long i = i0; i < d.g.size; i += stride) {
            double acc = xo[i];
            for (int k = 0; k < d.m; ++k) acc += d.dsc[k] * (double)Z[(long long)k * d.ld + i];
            xo[i] = acc;
        }
    }
}

template <typename T>
jfnk_status launch_bvec(BOp op, const BVec* dev_desc, const BItem* dev_items, int nitems, cudaStream_t st) {
    if (nitems <= 0) return JFNK_OK;
#define JFNK_BV(OPX)                                                                   \
    case OPX: bvec_kernel<T, OPX><<<nitems, kBThreads, 0, st>>>(dev_desc, dev_items); break;
    switch (op) {
        JFNK_BV(BOp::CAST_D2T)
        JFNK_BV(BOp::CAST_T2D)
        JFNK_BV(BOp::COPY_T)
        JFNK_BV(BOp::AXPBY_D)
        JFNK_BV(BOp::ADDSC_D)
        JFNK_BV(BOp::SCALE_INV_T)
        JFNK_BV(BOp::STAT)
        JFNK_BV(BOp::CHEB_START)
        JFNK_BV(BOp::RESTRICT)
        JFNK_BV(BOp::PROLONG_ADD)
        JFNK_BV(BOp::SPLITMIX)
        JFNK_BV(BOp::MDOT)
        JFNK_BV(BOp::MAXPY_SUB)
        JFNK_BV(BOp::COMBINE_T)
        JFNK_BV(BOp::CAST_SCALE_INT_D)
    }
#undef JFNK_BV
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}
template jfnk_status launch_bvec<float>(BOp, const BVec*, const BItem*, int, cudaStream_t);
template jfnk_status launch_bvec<double>(BOp, const BVec*, const BItem*, int, cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void bscalar_kernel(BScalar op, const BScal* __restrict__ descs, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const BScal& d = descs[i];
    if (op == BScalar::RATIO) {
        const double b = *d.x2;
        *d.out = b > 0.0 ? *d.x / b : 0.0;
    } else if (op == BScalar::CHEB_TABLE) {
        const double l = *d.x;
        if ((!(l > 0.0) || !isfinite(l)) && d.status) atomicOr(d.status, 2);
        double theta, c1, c2;
        cheb_coeffs(l, d.a, d.b, 0, theta, c1, c2);
        d.cheb->theta_inv = 1.0 / theta;
        d.cheb->theta_invf = (float)(1.0 / theta);
        for (int k = 0; k < d.m && k < kMaxChebDegree; ++k) {
            cheb_coeffs(l, d.a, d.b, k, theta, c1, c2);
            d.cheb->c1[k] = c1;
            d.cheb->c2[k] = c2;
            d.cheb->c1f[k] = (float)c1;
            d.cheb->c2f[k] = (float)c2;
        }
    } else if (op == BScalar::SET_EPS) {
        const double e = d.a;
        const double inv = e > 0.0 ? 1.0 / e : 0.0;
        d.slot->e = e;
        d.slot->inv = inv;
        d.slot->ef = (float)e;
        d.slot->invf = (float)inv;
    }
}

jfnk_status launch_bscalar(BScalar op, const BScal* dev_desc, int count, cudaStream_t st) {
    if (count <= 0) return JFNK_OK;
    bscalar_kernel<<<(count + 127) / 128, 128, 0, st>>>(op, dev_desc, count);
    JFNK_LAUNCH_CHECK();
    return JFNK_OK;
}

}  // namespace jfnk
