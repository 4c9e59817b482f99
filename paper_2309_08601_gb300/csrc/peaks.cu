// Throughput probes of the arithmetic pipes that bound this library's kernels (a measurement
// service for rooflines; the paper has no counterpart). Each probe fills every SM with work that
// only the probed pipe limits: independent chains of FP32 fused multiply-adds (one lane per
// instruction), of the packed two-lane FP32 FMA of sm_100 and later (__ffma2_rn) and of FP64 FMAs
// on register operands; and back-to-back tcgen05 tensor-core MMAs (BF16 and TF32 inputs, FP32
// accumulation) on operands resident in shared memory. The SM clock of the run is measured
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

// ---- tensor-core probe: one thread per CTA issues back-to-back tcgen05.mma (M = 128, N = 256,
// K = 16 BF16 or 8 TF32, FP32 accumulation in tensor memory) on operands resident in shared
// memory (every element 1/64, so the accumulator stays small), commits to an mbarrier, and the
// CTA waits for it (bounded, about a second) before freeing the tensor memory.
constexpr int kMmaM = 128, kMmaN = 256;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // canonical K-major layout without swizzle: start, leading (K) and stride (M/N) offsets
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

template <bool TF32>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int iters, unsigned long long* err, long long* cycles)
{
    __shared__ __align__(1024) uint32_t ops[3072];  // A: 128 rows x 32 B, B: 256 rows x 32 B
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long done;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t one64 = TF32 ? 0x3c800000u : 0x3c803c80u;  // 1/64 in FP32 / two BF16
    for (int i = tid; i < 3072; i += 128) ops[i] = one64;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kMmaN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&done)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const long long t0 = clock64();
    if (tid == 0) {
        constexpr uint32_t fmt = TF32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
                               ((uint32_t)(kMmaM >> 4) << 24);
        const uint64_t a = desc_noswizzle(smem_addr(ops), 128, 256);
        const uint64_t b = desc_noswizzle(smem_addr(ops + 1024), 128, 256);
        for (int i = 0; i < iters; ++i) {
            const uint32_t acc = i > 0 ? 1u : 0u;
            if constexpr (TF32)
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(a), "l"(b), "r"(idesc), "r"(acc));
            else
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(a), "l"(b), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&done))
                     : "memory");
    }
    // bounded wait for the commit (the MMAs take well under a millisecond)
    const long long w0 = clock64();
    bool ok = false;
    while (true) {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(r)
            : "r"(smem_addr(&done)), "r"(0)
            : "memory");
        if (r) {
            ok = true;
            break;
        }
        if (clock64() - w0 > (1LL << 31)) break;
    }
    if (!ok && tid == 0) atomicOr(err, 1ULL);
    if (blockIdx.x == 0 && tid == 0) *cycles = clock64() - t0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // the issue loop takes a few million cycles, so after a wait of 2^31 cycles no MMA is in
    // flight whatever the outcome: the tensor memory is always freed
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmaN));
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

// kinds 3 (BF16) and 4 (TF32): two CTAs per SM, each with its own accumulator; best of three
// timed launches after one warm-up
static mp3pcf_status mma_peak(bool tf32, cudaStream_t st, double* flops, double* mhz)
{
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MP3PCF_ECUDA;
    const int grid = 2 * n_sm, iters = 16384;
    // 96 KB of (unused) dynamic shared memory per CTA keeps at most two CTAs on an SM, so the two
    // 256-column tensor-memory allocations of an SM never wait for each other
    const size_t pad_smem = 96 * 1024;
    cudaError_t ea = cudaFuncSetAttribute(peaks::mma_probe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad_smem);
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(peaks::mma_probe_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad_smem);
    if (ea != cudaSuccess) return MP3PCF_ECUDA;
    unsigned long long* err = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&err, sizeof(unsigned long long)) != cudaSuccess) return MP3PCF_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) {
        cudaFree(err);
        return MP3PCF_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned long long), st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        if (tf32)
            peaks::mma_probe_kernel<true><<<grid, 128, pad_smem, st>>>(iters, err, cyc);
        else
            peaks::mma_probe_kernel<false><<<grid, 128, pad_smem, st>>>(iters, err, cyc);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, t);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    unsigned long long herr = 0;
    long long hcyc = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hcyc, cyc, sizeof(hcyc), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(err);
    cudaFree(cyc);
    if (e != cudaSuccess) return MP3PCF_ECUDA;
    if (herr) return MP3PCF_ETIMEOUT;
    const double k = tf32 ? 8.0 : 16.0;
    *flops = 2.0 * peaks::kMmaM * peaks::kMmaN * k * iters * grid / (best * 1e-3);
    // one CTA's cycles over its share of the launch (the two CTAs of an SM share its tensor core)
    if (mhz) *mhz = (double)hcyc / (best * 1e3);
    return MP3PCF_OK;
}

extern "C" mp3pcf_status mp3pcf_measure_peak(int32_t kind, void* stream, double* h_flops_per_s, double* h_sm_mhz)
{
    if (kind < 0 || kind > 4 || !h_flops_per_s) return MP3PCF_EINVAL;
    if (kind >= 3) return mma_peak(kind == 4, (cudaStream_t)stream, h_flops_per_s, h_sm_mhz);
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
