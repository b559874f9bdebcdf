// Arithmetic peaks of the GPU the library runs on, measured with independent
// FMA chains: the denominators of the element kernels' ALU rooflines (the FP64
// kernels are bound by the FP64 pipe, the FP32 ones by FP32 issue).  The paper
// has no counterpart; it measures nothing on GPUs.
#include <cuda_runtime.h>

#include "common.cuh"
#include "pf2.cuh"

namespace jfnk {

namespace {

constexpr int kChains = 8;         // independent accumulators per thread
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;

// written only when the accumulated value equals an impossible sentinel, so
// the chains cannot be removed as dead code and nothing is ever stored
__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_chain_kernel(int iters, T a, T b) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x & 7) * (T)0.125 + (T)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == (T)-1.5e30) g_probe_sink = (double)s;
}

__global__ void __launch_bounds__(kProbeThreads) fma_chain_f32x2_kernel(int iters, float a, float b) {
    pf2 acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = pf2_pack((float)(threadIdx.x & 7) * 0.125f + k, (float)k - 0.5f);
    const pf2 pa = pf2_pack(a, a), pb = pf2_pack(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = madd(acc[k], pa, pb);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        pf2_unpack(acc[k], lo, hi);
        s += lo + hi;
    }
    if (s == -1.5e30f) g_probe_sink = (double)s;
}

// FMA per second of one launch doing `fmas` FMA operations (best of `reps`
// after one warm-up launch).
template <typename Launch>
jfnk_status time_probe(Launch launch, double fmas, int reps, cudaStream_t st, double* rate) {
    cudaEvent_t e0, e1;
    JFNK_CUDA_TRY(cudaEventCreate(&e0));
    JFNK_CUDA_TRY(cudaEventCreate(&e1));
    launch();
    JFNK_LAUNCH_CHECK();
    float best = 0.0f;
    for (int r = 0; r < reps; ++r) {
        JFNK_CUDA_TRY(cudaEventRecord(e0, st));
        launch();
        JFNK_LAUNCH_CHECK();
        JFNK_CUDA_TRY(cudaEventRecord(e1, st));
        JFNK_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        JFNK_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (r == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *rate = best > 0.0f ? fmas / (best * 1e-3) : 0.0;
    return JFNK_OK;
}

}  // namespace

}  // namespace jfnk

jfnk_status jfnk_measure_peaks(double* fp64_fma_per_s, double* fp32_fma_per_s, double* fp32x2_fma_per_s,
                               void* stream) {
    using namespace jfnk;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    JFNK_CUDA_TRY(cudaGetDevice(&dev));
    JFNK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * kProbeBlocksPerSM;
    const double threads = (double)blocks * kProbeThreads;
    // chain lengths for launches of roughly 10-30 ms at the expected rates
    const int it64 = 5000, it32 = 300000, it32x2 = 200000;
    if (fp64_fma_per_s) {
        JFNK_TRY(time_probe([&] { fma_chain_kernel<double><<<blocks, kProbeThreads, 0, st>>>(it64, 0.999999, 1e-7); },
                            threads * it64 * kChains, 3, st, fp64_fma_per_s));
    }
    if (fp32_fma_per_s) {
        JFNK_TRY(time_probe([&] { fma_chain_kernel<float><<<blocks, kProbeThreads, 0, st>>>(it32, 0.9999f, 1e-4f); },
                            threads * it32 * kChains, 3, st, fp32_fma_per_s));
    }
    if (fp32x2_fma_per_s) {
        JFNK_TRY(time_probe([&] { fma_chain_f32x2_kernel<<<blocks, kProbeThreads, 0, st>>>(it32x2, 0.9999f, 1e-4f); },
                            threads * it32x2 * kChains * 2, 3, st, fp32x2_fma_per_s));
    }
    return JFNK_OK;
}
