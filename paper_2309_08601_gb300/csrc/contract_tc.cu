// Stage (b) on the 5th-generation tensor cores (tcgen05): the multipole components
// Upsilon_{mu,n}(b1,b2) and N_n(b1,b2) as real GEMMs over the centre-galaxy axis (paper
// Sec. 3.1, Eqs. Upsilon0_Derivation, Upsilon1-3, 3PCF_Normalization, tomoGn).
//
// A group g = (Z-triplet, component, order n) is the complex product sum_i L_i(b1) R_i(b2) with
// L = c_i X_i (c_i = -w gamma, -(w gamma)^*, or w) and R = Y_i. Written in reals, the rows
// (Re L(b1), Im L(b1)) times the columns (Re R(b2), Im R(b2)) give four blocks whose
// combination is the complex result. Up to 128 / (2 n_bins) groups are stacked along M = 128
// (their right operands along N); only the diagonal blocks are kept.
//
// Split precision: every operand value x is written as hi + lo with hi = round(x) and
// lo = round(x - hi) in BF16 (or TF32), and D += A_hi B_hi + A_hi B_lo + A_lo B_hi is
// accumulated in FP32 in tensor memory (the lo*lo term is below the rounding of the others).
// The tensor core's FP32 accumulation is not round-to-nearest: over thousands of centres its
// error grows with the number of accumulating MMAs (measured: 1e-4 relative after ~1700 BF16 or
// ~3400 TF32 MMAs, TF32 worse). So every kFlush stages the accumulator is read out (tcgen05.ld)
// and added to FP32 block sums in shared memory by the CUDA cores, and restarted: no chain is
// longer than 3 kFlush KT / KI MMAs.
//
// Pipeline per CTA (one tile of groups, one slice of the centre axis): all threads stage the
// operands of KT centres into one of two shared-memory stages in the canonical no-swizzle
// K-major layout (8-row x 16-byte core matrices), one thread issues the MMAs of that stage and
// commits them to the stage's mbarrier, and the threads go on staging the other stage while the
// tensor core works. Every wait on an mbarrier is bounded (about a second); a wait that gives
// up sets bit 2 of the error word, stops the issue of further MMAs, waits (bounded) for those in
// flight and frees the tensor memory. The per-slice FP32 sums are written as FP64 partials and
// summed in a fixed order by contract_reduce_kernel, so results are deterministic.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace mp3 {

namespace tc {

constexpr int kThreads = 256;  // 8 warps: two per TMEM lane quarter
constexpr int kM = 128;         // MMA rows (TMEM lanes)
constexpr int kMaxGroups = 8;   // groups stacked in one tile
constexpr int kTmemCols = 128;  // FP32 accumulator columns (N <= 128)
constexpr int kFlush = 8;       // tiles per tensor-core accumulation chain

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, int parity, unsigned long long* err)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) {
            if (err) atomicOr(err, 2ULL);
            return false;
        }
    }
}

// the two split-precision forms: element size, centres per stage, K per MMA, operand format
struct Bf16Split {
    static constexpr int ES = 2;
    static constexpr int KT = 32;
    static constexpr int KI = 16;
    static constexpr uint32_t FMT = 1;
    // hi and lo parts of two values packed as (first, second) in one 32-bit word each
    __device__ static void split2(float x0, float x1, uint32_t& hi, uint32_t& lo)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
    __device__ static void split1(float, uint32_t&, uint32_t&) {}
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
    {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
};

struct Tf32Split {
    static constexpr int ES = 4;
    static constexpr int KT = 16;
    static constexpr int KI = 8;
    static constexpr uint32_t FMT = 2;
    __device__ static uint32_t to_tf32(float x)
    {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return r;
    }
    __device__ static void split2(float, float, uint32_t&, uint32_t&) {}
    __device__ static void split1(float x, uint32_t& hi, uint32_t& lo)
    {
        hi = to_tf32(x);
        lo = to_tf32(x - __uint_as_float(hi));
    }
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
    {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
};

struct TcArgs {
    ContractArgs<float> c;
    int groups;   // nz^3 * groups_per_zt(n_max)
    int gt;       // groups per tile
    int npad;     // MMA N: gt * 2 nb rounded up to 16
    unsigned long long* err;
};

// one stage: A_hi, A_lo, B_hi, B_lo, each 128 rows x KT centres in the canonical no-swizzle
// K-major layout: element (r, k) at ((r/8)*(KT/T) + k/T)*128 B + (r%8)*16 B + (k%T)*ES
template <class SP>
struct Layout {
    static constexpr int T = 16 / SP::ES;                 // elements per 16-byte core row
    static constexpr int KT = SP::KT;
    static constexpr int SBO = (KT / T) * 128;            // bytes between 8-row core groups
    static constexpr int OP_BYTES = kM * KT * SP::ES;
    static constexpr int STAGE_BYTES = 4 * OP_BYTES;
    static constexpr int PK = 4 / SP::ES;                 // centres per 32-bit word
    static constexpr int KW = KT / PK;                    // 32-bit words along K per row
    __device__ static uint32_t word_off(int r, int kw)
    {
        // kw-th 32-bit word of row r: centres kw*PK .. kw*PK + PK - 1
        return (uint32_t)((r / 8) * SBO + (kw / 4) * 128 + (r % 8) * 16 + (kw % 4) * 4);
    }
};

struct GroupInfo {
    int z1, z2, z3, kind, mx, my;
};

// FP32 sums of the diagonal blocks in shared memory: dacc[t][i][j], i, j in [0, 2 nb)
__device__ __forceinline__ int dacc_size(int ng, int nb) { return ng * 4 * nb * nb; }

template <class SP>
__global__ void __launch_bounds__(kThreads) contract_tc_kernel(const TcArgs a)
{
    using L = Layout<SP>;
    constexpr int KT = SP::KT;
    constexpr int PK = L::PK;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ float4 coef_sm[KT];  // per centre of the stage: (w gamma_1, w gamma_2, w, zbin)
    __shared__ GroupInfo gi[kMaxGroups];

    const ContractArgs<float>& A = a.c;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const int nbb = nb * nb, nb2 = 2 * nb;
    const int g0 = blockIdx.x * a.gt;
    const int ng = min(a.gt, a.groups - g0);
    const int sl = blockIdx.y, slices = gridDim.y;
    const int per = (A.n_centres + slices - 1) / slices;
    const int c0 = min(A.n_centres, sl * per), c1 = min(A.n_centres, c0 + per);
    const int ntiles = (c1 - c0 + KT - 1) / KT;
    const int MG = 2 * n_max + 3, MW = 2 * n_max + 1;
    float* dacc = reinterpret_cast<float*>(smem + 2 * L::STAGE_BYTES);

    if (tid < ng) {
        const int per_zt = groups_per_zt(n_max);
        const int g = g0 + tid;
        const int zt = g / per_zt, loc = g % per_zt;
        GroupInfo q;
        q.z1 = zt / (nz * nz);
        q.z2 = (zt / nz) % nz;
        q.z3 = zt % nz;
        int n;
        if (loc < 4 * (n_max + 1)) {
            q.kind = loc / (n_max + 1);
            n = loc % (n_max + 1);
        } else {
            q.kind = 4;
            n = loc - 4 * (n_max + 1);
        }
        // orders of the first (X) and second (Y) moment, as in the SIMT form
        switch (q.kind) {
            case 0: q.mx = n - 3; q.my = -n - 3; break;   // G_{n-3} G_{-n-3}
            case 1: q.mx = n - 1; q.my = -n - 1; break;   // G_{n-1} G_{-n-1}
            case 2: q.mx = -n - 1; q.my = -n - 3; break;  // G_{-n-1}^* G_{-n-3}
            case 3: q.mx = n - 3; q.my = n - 1; break;    // G_{n-3} G_{n-1}^*
            default: q.mx = n; q.my = n; break;           // W_n W_n^*
        }
        gi[tid] = q;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero both stages (rows outside the stacked groups stay zero) and the block sums
    const int zero16 = (2 * L::STAGE_BYTES + dacc_size(ng, nb) * 4 + 15) / 16;
    for (int i = tid; i < zero16; i += kThreads) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | (SP::FMT << 7) | (SP::FMT << 10) | ((uint32_t)(a.npad >> 3) << 17) |
                           ((uint32_t)(kM >> 4) << 24);
    const int TB = ng * nb;
    const int items = L::KW * TB;

    // TMEM lane quarter and column half this warp reads; the accumulator row it holds
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const int rt = row / nb2, ri = row % nb2;  // group and row within the group's block
    const int ncol = a.npad / 2, colb = half * ncol;

    // adds the accumulator (the sums of the tiles since the last flush) to dacc, after the MMAs
    // of tile t completed; false if the bounded wait gave up
    auto flush = [&](int t) -> bool {
        const bool done = mbar_wait(smem_u32(&mbar[t & 1]), (t >> 1) & 1, a.err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, done)) {
            for (int col = colb; col < colb + ncol; col += 8) {
                uint32_t r[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                               "=r"(r[6]), "=r"(r[7])
                             : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (rt < ng) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int cj = col + j - rt * nb2;
                        if (cj >= 0 && cj < nb2) dacc[(rt * nb2 + ri) * nb2 + cj] += __uint_as_float(r[j]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        const bool all = __syncthreads_and(done);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return all;
    };

    int issued = 0;
    bool ok = true;
    for (int tile = 0; tile < ntiles; ++tile) {
        const int st = tile & 1;
        unsigned char* sbase = smem + st * L::STAGE_BYTES;
        // the stage is free once the MMAs issued on it two tiles ago have completed
        bool good = true;
        if (tid == 0 && tile >= 2) good = mbar_wait(smem_u32(&mbar[st]), ((tile - 2) >> 1) & 1, a.err);
        const int cb = c0 + tile * KT;
        if (tid < KT) {
            const int c = cb + tid;
            float4 cf = make_float4(0.f, 0.f, 0.f, -1.f);
            if (c < c1) {
                const int d = A.centre_idx[c];
                const Pay<float> pv = A.pay[d];
                cf = make_float4(pv.a, pv.b, pv.w, (float)(A.zs ? (int)A.zs[d] : 0));
            }
            coef_sm[tid] = cf;
        }
        if (!__syncthreads_and(good)) {
            ok = false;
            break;
        }

        // item = (word column kw, group t, bin b); 4 consecutive lanes fill one 16-byte core
        // row, 8 lane quads fill 8 different rows: conflict-free 32-bit stores
        for (int it = tid; it < items; it += kThreads) {
            const int kw_lo = it & 3, rest = it >> 2;
            const int tb = rest % TB, kw = (rest / TB) * 4 + kw_lo;
            const int t = tb / nb, b = tb % nb;
            const GroupInfo q = gi[t];
            const bool isW = q.kind == 4;
            const cx<float>* src = isW ? A.W : A.G;
            const int M = isW ? MW : MG, off = isW ? 0 : n_max + 3;
            float xr[PK], xi[PK], yr[PK], yi[PK];
#pragma unroll
            for (int p = 0; p < PK; ++p) {
                const int k = kw * PK + p, c = cb + k;
                const float4 cf = coef_sm[k];
                cx<float> X{0.f, 0.f}, Y{0.f, 0.f};
                if (c < c1 && (int)cf.w == q.z1) {
                    const float2 xv = __ldg(reinterpret_cast<const float2*>(
                        src + (((size_t)c * nz + q.z2) * nb + b) * M + q.mx + off));
                    const float2 yv = __ldg(reinterpret_cast<const float2*>(
                        src + (((size_t)c * nz + q.z3) * nb + b) * M + q.my + off));
                    X = {xv.x, xv.y};
                    Y = {yv.x, yv.y};
                    if (q.kind == 2) X = cconj(X);
                    if (q.kind >= 3) Y = cconj(Y);
                    cx<float> co;
                    if (isW)
                        co = {cf.z, 0.f};
                    else if (q.kind == 1)
                        co = {-cf.x, cf.y};  // -(w gamma)^*
                    else
                        co = {-cf.x, -cf.y};  // -(w gamma)
                    X = cmul(co, X);
                }
                xr[p] = X.x;
                xi[p] = X.y;
                yr[p] = Y.x;
                yi[p] = Y.y;
            }
            uint32_t h[4], l[4];
            if constexpr (PK == 2) {
                SP::split2(xr[0], xr[PK - 1], h[0], l[0]);
                SP::split2(xi[0], xi[PK - 1], h[1], l[1]);
                SP::split2(yr[0], yr[PK - 1], h[2], l[2]);
                SP::split2(yi[0], yi[PK - 1], h[3], l[3]);
            } else {
                SP::split1(xr[0], h[0], l[0]);
                SP::split1(xi[0], h[1], l[1]);
                SP::split1(yr[0], h[2], l[2]);
                SP::split1(yi[0], h[3], l[3]);
            }
            const int rre = t * nb2 + b, rim = rre + nb;
            const uint32_t ore = L::word_off(rre, kw), oim = L::word_off(rim, kw);
            *reinterpret_cast<uint32_t*>(sbase + 0 * L::OP_BYTES + ore) = h[0];
            *reinterpret_cast<uint32_t*>(sbase + 1 * L::OP_BYTES + ore) = l[0];
            *reinterpret_cast<uint32_t*>(sbase + 0 * L::OP_BYTES + oim) = h[1];
            *reinterpret_cast<uint32_t*>(sbase + 1 * L::OP_BYTES + oim) = l[1];
            *reinterpret_cast<uint32_t*>(sbase + 2 * L::OP_BYTES + ore) = h[2];
            *reinterpret_cast<uint32_t*>(sbase + 3 * L::OP_BYTES + ore) = l[2];
            *reinterpret_cast<uint32_t*>(sbase + 2 * L::OP_BYTES + oim) = h[3];
            *reinterpret_cast<uint32_t*>(sbase + 3 * L::OP_BYTES + oim) = l[3];
        }
        // make the generic-proxy stores visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // every kFlush tiles the accumulator is added to the FP32 block sums and restarted, so
        // no tensor-core accumulation chain is longer than 3 kFlush (KT / KI) MMAs
        bool fresh = tile == 0;
        if (tile > 0 && tile % kFlush == 0) {
            if (!flush(tile - 1)) {
                ok = false;
                break;
            }
            fresh = true;
        }
        if (tid == 0) {
            const uint32_t s0 = smem_u32(sbase);
#pragma unroll
            for (int kk = 0; kk < KT / SP::KI; ++kk) {
                const uint32_t ko = kk * 256;  // two core matrices along K per MMA
                const uint64_t ah = smem_desc(s0 + 0 * L::OP_BYTES + ko, 128, L::SBO);
                const uint64_t al = smem_desc(s0 + 1 * L::OP_BYTES + ko, 128, L::SBO);
                const uint64_t bh = smem_desc(s0 + 2 * L::OP_BYTES + ko, 128, L::SBO);
                const uint64_t bl = smem_desc(s0 + 3 * L::OP_BYTES + ko, 128, L::SBO);
                SP::mma(tmem, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
                SP::mma(tmem, ah, bl, idesc, 1u);
                SP::mma(tmem, al, bh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
        issued = tile + 1;
    }

    if (ok && ntiles > 0) {
        ok = flush(ntiles - 1);
    } else if (issued > 0) {
        // a wait gave up: wait (bounded) for this thread's last commit, which tracks all MMAs
        if (tid == 0) mbar_wait(smem_u32(&mbar[(issued - 1) & 1]), ((issued - 1) >> 1) & 1, a.err);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    // diagonal blocks: (Re L Re R - Im L Im R, Re L Im R + Im L Re R), in FP64
    for (int it = tid; it < ng * nbb; it += kThreads) {
        const int t = it / nbb, o = it % nbb, b1 = o / nb, b2 = o % nb;
        double re = 0.0, im = 0.0;
        if (ok) {
            const float* D = dacc + t * nb2 * nb2;
            re = (double)D[b1 * nb2 + b2] - (double)D[(nb + b1) * nb2 + nb + b2];
            im = (double)D[b1 * nb2 + nb + b2] + (double)D[(nb + b1) * nb2 + b2];
        }
        double* dst = A.partial + 2 * (((size_t)sl * a.groups + (g0 + t)) * nbb + o);
        dst[0] = re;
        dst[1] = im;
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

template <class SP>
static size_t smem_bytes(int gt, int nb)
{
    return 2 * (size_t)Layout<SP>::STAGE_BYTES + (size_t)gt * 4 * nb * nb * sizeof(float);
}

// slices of the centre axis: fill the resident CTA slots in whole waves, at least 4 stages
// of centres per slice, at most 64 slices
static int pick_slices(int tiles, int slots, int64_t n_centres, int kt)
{
    const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(64, n_centres / (4 * kt)));
    int best = 1;
    double best_score = -1.0;
    for (int s = 1; s <= smax; ++s) {
        const int64_t ctas = (int64_t)tiles * s;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        const double score = eff - 0.002 * s;
        if (score > best_score) {
            best_score = score;
            best = s;
        }
    }
    return best;
}

template <class SP>
static cudaError_t launch_tc(TcArgs a, int n_sm, int* splits_out, bool plan_only, cudaStream_t st)
{
    const size_t smem = smem_bytes<SP>(a.gt, a.c.nb);
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, contract_tc_kernel<SP>, kThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, 512 / kTmemCols));
    const int tiles = (a.groups + a.gt - 1) / a.gt;
    const int slices = pick_slices(tiles, per_sm * n_sm, a.c.n_centres, SP::KT);
    *splits_out = slices;
    if (plan_only) return cudaSuccess;
    if (slices != a.c.splits) return cudaErrorInvalidValue;  // partial buffer sized for another plan
    contract_tc_kernel<SP><<<dim3(tiles, slices), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tc

cudaError_t launch_contract_tc(const ContractArgs<float>& c, bool tf32, int n_sm, unsigned long long* err,
                               int* splits, bool plan_only, cudaStream_t st)
{
    tc::TcArgs a;
    a.c = c;
    a.groups = c.nz * c.nz * c.nz * groups_per_zt(c.n_max);
    a.gt = std::min(tc::kMaxGroups, tc::kM / (2 * c.nb));
    if (a.gt < 1) return cudaErrorInvalidValue;
    a.npad = ((a.gt * 2 * c.nb + 15) / 16) * 16;
    a.err = err;
    return tf32 ? tc::launch_tc<tc::Tf32Split>(a, n_sm, splits, plan_only, st)
                : tc::launch_tc<tc::Bf16Split>(a, n_sm, splits, plan_only, st);
}

}  // namespace mp3
