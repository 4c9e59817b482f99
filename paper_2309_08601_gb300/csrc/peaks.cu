// Throughput probes of the arithmetic pipes that bound this library's kernels (a measurement
// service for rooflines; the paper has no counterpart). Each probe fills every SM with warps that
// run independent chains of one instruction kind on register operands, so the pipe, not latency
// or memory, limits it: FP32 fused multiply-add (one lane per instruction), the packed two-lane
// FP32 FMA of sm_100 and later (__ffma2_rn), and FP64 FMA. The SM clock of the run is measured
// alongside: one block's clock64 cycles over the global timer's nanoseconds for the same span.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace mp3 {

namespace peaks {

constexpr int kThreads = 256;
constexpr int kChains = 16;     // independent accumulation chains per thread

template <int KIND>
__global__ void __launch_bounds__(kThreads) probe_kernel(float mf, float af, double md, double ad, int iters,
                                                         float* sink, long long* cycles)
{
    const long long t0 = clock64();
    unsigned long long g0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    if constexpr (KIND == 0) {
        float v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
#pragma unroll 4
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], mf, af);
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += v[c];
        if (s == -1.0f) sink[threadIdx.x] = s;  // never true for the probe's operands
    } else if constexpr (KIND == 1) {
        float2 v[kChains];
        const float2 m2 = make_float2(mf, mf), a2 = make_float2(af, af);
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = make_float2((float)(threadIdx.x + c), (float)c);
#pragma unroll 4
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], m2, a2);
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
        if (s == -1.0f) sink[threadIdx.x] = s;
    } else {
        double v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = (double)(threadIdx.x + c);
#pragma unroll 4
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], md, ad);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += v[c];
        if (s == -1.0) sink[threadIdx.x] = (float)s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long t1 = clock64();
        unsigned long long g1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
        cycles[0] = t1 - t0;
        cycles[1] = (long long)(g1 - g0);
    }
}

template <int KIND>
static cudaError_t run(int grid, int iters, cudaStream_t st, float* sink, long long* cyc, float* ms)
{
    // operands that keep every chain finite and normal: v <- v * (1 - 2^-20) + 2^-10
    const float mf = 1.0f - 1.0f / 1048576.0f, af = 1.0f / 1024.0f;
    const double md = 1.0 - 1.0 / 1048576.0, ad = 1.0 / 1024.0;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        probe_kernel<KIND><<<grid, kThreads, 0, st>>>(mf, af, md, ad, iters, sink, cyc);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, t);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace peaks

}  // namespace mp3

using namespace mp3;

extern "C" mp3pcf_status mp3pcf_measure_peak(int32_t kind, void* stream, double* h_flops_per_s, double* h_sm_mhz)
{
    if (kind < 0 || kind > 2 || !h_flops_per_s) return MP3PCF_EINVAL;
    int dev = 0, n_sm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MP3PCF_ECUDA;
    cudaError_t e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peaks::probe_kernel<0>, peaks::kThreads, 0)
                    : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peaks::probe_kernel<1>, peaks::kThreads, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peaks::probe_kernel<2>, peaks::kThreads, 0);
    if (e != cudaSuccess) return MP3PCF_ECUDA;
    const int waves = 2;
    const int grid = n_sm * std::max(per_sm, 1) * waves;
    // dependent steps per chain: about 0.1-0.3 s per launch on every pipe (FP64 is ~1/64 of FP32)
    const int iters = kind == 2 ? 16 : 1024;
    float* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * peaks::kThreads) != cudaSuccess) return MP3PCF_ENOMEM;
    if (cudaMalloc(&cyc, 2 * sizeof(long long)) != cudaSuccess) {
        cudaFree(sink);
        return MP3PCF_ENOMEM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float ms = 0.0f;
    e = kind == 0 ? peaks::run<0>(grid, iters, st, sink, cyc, &ms)
        : kind == 1 ? peaks::run<1>(grid, iters, st, sink, cyc, &ms)
                    : peaks::run<2>(grid, iters, st, sink, cyc, &ms);
    long long cycles[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(cycles, cyc, sizeof(cycles), cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess) return MP3PCF_ECUDA;
    // FMAs per thread: chains x steps, two lanes each for the packed form; 2 flops per FMA
    const double fmas = (double)grid * peaks::kThreads * peaks::kChains * iters * (kind == 1 ? 2.0 : 1.0);
    *h_flops_per_s = 2.0 * fmas / (ms * 1e-3);
    // cycles per nanosecond of one block of the last launch
    if (h_sm_mhz) *h_sm_mhz = cycles[1] > 0 ? 1e3 * (double)cycles[0] / (double)cycles[1] : 0.0;
    return MP3PCF_OK;
}
