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
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace mp3 {

namespace tc {

constexpr int kConvWarps = 16;                 // converter warps: four per TMEM lane quarter
constexpr int kThreads = (kConvWarps + 2) * 32;  // + one TMA warp + one MMA warp
constexpr int kM = 128;         // MMA rows (TMEM lanes)
constexpr int kMaxGroups = 8;   // groups stacked in one tile
constexpr int kTmemCols = 128;  // FP32 columns of one accumulator (N <= 128); two accumulators
constexpr int kFlush = 32;      // tiles per tensor-core accumulation chain
constexpr int kStages = 2;      // operand stages

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
    static constexpr int KT = 16;
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
    static constexpr int KT = 8;
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
    int groups;   // nz^3 * groups_per_zt(n_max): index space of the partial sums
    int gt;       // groups per tile
    int npad;     // MMA N: gt * 2 nb rounded up to 32 (8 TMEM columns per converter part and load)
    int nbp;      // bins padded to even (the moment rows)
    int ta, tw;   // tiles per component of Upsilon (n_max + 1 orders) and of N (2 n_max + 1 orders)
    int fixed_slices;  // > 0: this many centre slices instead of the automatic choice
    int skip_copies;   // test hook: issue no TMA copies, so every wait on them runs out
    unsigned long long* err;
};

// TMA boxes of one raw slot: X moments [gt orders][KT centres][nbp bins] complex, Y moments
// (same), coefficients [KT]
struct RawLayout {
    int box_bytes, slot_bytes;
    __host__ __device__ RawLayout(int kt, int nbp, int gt)
    {
        box_bytes = gt * kt * nbp * 8;
        slot_bytes = ((2 * box_bytes + kt * 16) + 127) / 128 * 128;
    }
};

// one operand stage: A_hi, A_lo, B_hi, B_lo, each 128 rows x KT centres in the canonical no-swizzle
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

constexpr int kRaw = 3;  // raw slots: the TMA copies run two stages ahead of the conversion

template <class SP>
static size_t smem_bytes(int kt, int nb, int nbp, int gt)
{
    const RawLayout R(kt, nbp, gt);
    return (size_t)kRaw * R.slot_bytes + kStages * (size_t)Layout<SP>::STAGE_BYTES + (size_t)gt * 4 * nb * nb * sizeof(float);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, int parity, volatile int* abort, unsigned long long* err)
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
        if (*abort) return false;
        if (clock64() - t0 > (1LL << 31)) {
            if (err) atomicOr(err, 2ULL);
            *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// agreement among the converter warps only (named barrier 1); every converter thread reaches
// each of them, also after an abort, so none can wait for a warp that left

__device__ __forceinline__ bool conv_all(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kConvWarps * 32)
        : "memory");
    return r != 0;
}

// Grid: x = tiles of groups (a tile never spans two components or Z-triplets, so its orders are
// consecutive), y = slices of the centre axis. Warp roles: warps 0..kConvWarps-1 convert raw
// moments into split operands and flush the accumulators; warp kConvWarps issues the TMA copies;
// warp kConvWarps+1 issues the MMAs. They synchronise only through mbarriers:
//   rawfull[i]  (TMA bytes) -> converters     rawempty[i] (converter warps) -> TMA warp
//   opfull[j]   (converter warps) -> MMA warp opempty[j]  (MMA commit) -> converters
//   accfull[a]  (MMA commit) -> converters    accempty[a] (converter warps) -> MMA warp
template <class SP>
__global__ void __launch_bounds__(kThreads, 2) contract_tc_kernel(const __grid_constant__ CUtensorMap mapG,
                                                               const __grid_constant__ CUtensorMap mapW,
                                                               const __grid_constant__ CUtensorMap mapC,
                                                               const TcArgs a)
{
    using L = Layout<SP>;
    constexpr int KT = SP::KT;
    constexpr int PK = L::PK;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long rawfull[kRaw], rawempty[kRaw], opfull[kStages], opempty[kStages],
        accfull[2], accempty[2];
    __shared__ volatile int abort_flag;
    __shared__ int last_tma, last_mma;

    const ContractArgs<float>& A = a.c;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const int nbb = nb * nb, nb2 = 2 * nb, nbp = a.nbp;

    // ---- the tile: Z-triplet, component, first order, number of groups
    const int per_tile_zt = 4 * a.ta + a.tw;
    const int zt = blockIdx.x / per_tile_zt, r = blockIdx.x % per_tile_zt;
    int kind, n0, ng;
    if (r < 4 * a.ta) {
        kind = r / a.ta;
        n0 = (r % a.ta) * a.gt;
        ng = min(a.gt, n_max + 1 - n0);
    } else {
        kind = 4;
        n0 = (r - 4 * a.ta) * a.gt;
        ng = min(a.gt, 2 * n_max + 1 - n0);
    }
    const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
    const int gbase = zt * groups_per_zt(n_max) + (kind < 4 ? kind * (n_max + 1) : 4 * (n_max + 1)) + n0;
    // orders of group t: X m = ax + sx t, Y m = ay + sy t (as in the SIMT form)
    int ax, sx, ay, sy;
    switch (kind) {
        case 0: ax = n0 - 3; sx = 1; ay = -n0 - 3; sy = -1; break;   // G_{n-3} G_{-n-3}
        case 1: ax = n0 - 1; sx = 1; ay = -n0 - 1; sy = -1; break;   // G_{n-1} G_{-n-1}
        case 2: ax = -n0 - 1; sx = -1; ay = -n0 - 3; sy = -1; break; // G_{-n-1}^* G_{-n-3}
        case 3: ax = n0 - 3; sx = 1; ay = n0 - 1; sy = 1; break;     // G_{n-3} G_{n-1}^*
        default: ax = n0; sx = 1; ay = n0; sy = 1; break;            // W_n W_n^*
    }
    const int off = kind < 4 ? n_max + 3 : 0;
    // first order slot of each box: the lowest one of the tile
    const int ix0 = (sx > 0 ? ax : ax - (ng - 1)) + off;
    const int iy0 = (sy > 0 ? ay : ay - (ng - 1)) + off;
    const CUtensorMap* mapM = kind < 4 ? &mapG : &mapW;

    // slices of the centres of z-bin z1 (a contiguous range of the z-sorted centre list)
    const int sl = blockIdx.y, slices = gridDim.y;
    const int zc0 = A.zrange ? A.zrange[z1] : 0, zc1 = A.zrange ? A.zrange[z1 + 1] : A.n_centres;
    const int per = (zc1 - zc0 + slices - 1) / slices;
    const int c0 = min(zc1, zc0 + sl * per), c1 = min(zc1, c0 + per);
    const int ntiles = (c1 - c0 + KT - 1) / KT;
    const int nchains = (ntiles + kFlush - 1) / kFlush;

    const RawLayout R(KT, nbp, a.gt);
    unsigned char* raw = smem;
    unsigned char* ops = smem + kRaw * R.slot_bytes;
    // FP32 sums of the diagonal blocks: dq[gc][ri] = D[row of group gc / nb2, ri][gc], gc < ng nb2
    float* dq = reinterpret_cast<float*>(ops + kStages * L::STAGE_BYTES);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < kRaw; ++i) {
            mbar_init(smem_u32(&rawfull[i]), 1);
            mbar_init(smem_u32(&rawempty[i]), kConvWarps);
        }
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_u32(&opfull[i]), kConvWarps);
            mbar_init(smem_u32(&opempty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&accfull[i]), 1);
            mbar_init(smem_u32(&accempty[i]), kConvWarps);
        }
        abort_flag = 0;
        last_tma = 0;
        last_mma = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero the operand stages (rows outside the stacked groups stay zero) and the block sums
    {
        uint4* z = reinterpret_cast<uint4*>(ops);
        const int n16 = (kStages * L::STAGE_BYTES + ng * 4 * nbb * 4 + 15) / 16;
        for (int i = tid; i < n16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == kConvWarps) {
        // ================= TMA warp: copies of tile s into raw slot s % kRaw
        if (lane == 0) {
            const uint32_t tx_bytes = 2 * R.box_bytes + KT * 16;
            for (int s = 0; s < ntiles; ++s) {
                const int slot = s % kRaw;
                if (s >= kRaw && !wait_or_abort(smem_u32(&rawempty[slot]), ((s / kRaw) - 1) & 1, &abort_flag, a.err))
                    break;
                if (a.skip_copies) continue;
                const uint32_t dst = smem_u32(raw + slot * R.slot_bytes);
                const uint32_t bar = smem_u32(&rawfull[slot]);
                const int cb = c0 + s * KT;
                mbar_expect_tx(bar, tx_bytes);
                tma_load_4d(dst, mapM, 0, z2, cb, ix0, bar);
                tma_load_4d(dst + R.box_bytes, mapM, 0, z3, cb, iy0, bar);
                tma_load_2d(dst + 2 * R.box_bytes, &mapC, 0, cb, bar);
                last_tma = s + 1;
            }
        }
    } else if (warp == kConvWarps + 1) {
        // ================= MMA warp: three split products per K-step into accumulator chain % 2
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (SP::FMT << 7) | (SP::FMT << 10) |
                                   ((uint32_t)(a.npad >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            for (int s = 0; s < ntiles; ++s) {
                const int st = s % kStages, c = s / kFlush;
                const bool first = s % kFlush == 0;
                if (first && c >= 2 &&
                    !wait_or_abort(smem_u32(&accempty[c & 1]), ((c >> 1) - 1) & 1, &abort_flag, a.err))
                    break;
                if (!wait_or_abort(smem_u32(&opfull[st]), (s / kStages) & 1, &abort_flag, a.err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)((c & 1) * kTmemCols);
                const uint32_t s0 = smem_u32(ops + st * L::STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < KT / SP::KI; ++kk) {
                    const uint32_t ko = kk * 256;  // two core matrices along K per MMA
                    const uint64_t ah = smem_desc(s0 + 0 * L::OP_BYTES + ko, 128, L::SBO);
                    const uint64_t al = smem_desc(s0 + 1 * L::OP_BYTES + ko, 128, L::SBO);
                    const uint64_t bh = smem_desc(s0 + 2 * L::OP_BYTES + ko, 128, L::SBO);
                    const uint64_t bl = smem_desc(s0 + 3 * L::OP_BYTES + ko, 128, L::SBO);
                    SP::mma(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
                    SP::mma(d, ah, bl, idesc, 1u);
                    SP::mma(d, al, bh, idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&opempty[st]))
                             : "memory");
                if (s % kFlush == kFlush - 1 || s == ntiles - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&accfull[c & 1]))
                                 : "memory");
                last_mma = s + 1;
            }
        }
    } else {
        // ================= converter warps
        // this thread's conversion items, the same in every stage: item = (word column kw, group
        // t, bin b); 4 consecutive lanes fill one 16-byte core row, 8 lane quads fill 8 rows
        constexpr int kItems = (8 * 64 + kConvWarps * 32 - 1) / (kConvWarps * 32);  // KW * ng * nb <= 8 * 64
        const int TB = ng * nb;
        const int items = L::KW * TB;
        uint32_t i_ore[kItems], i_oim[kItems];
        int i_xo[kItems], i_yo[kItems], i_k[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const int it = tid + q * kConvWarps * 32;
            const int kw_lo = it & 3, rest = it >> 2;
            const int tb = rest % TB, kw = (rest / TB) * 4 + kw_lo;
            const int t = tb / nb, b = tb % nb;
            const int ox = ax + sx * t + off - ix0, oy = ay + sy * t + off - iy0;  // order plane in the box
            const int rre = t * nb2 + b;
            i_ore[q] = L::word_off(rre, kw);
            i_oim[q] = L::word_off(rre + nb, kw);
            i_k[q] = it < items ? kw * PK : 1 << 20;  // first centre of the word; out of range: no item
            i_xo[q] = (ox * KT + kw * PK) * nbp + b;  // complex index in the X box
            i_yo[q] = (oy * KT + kw * PK) * nbp + b;
        }
        // L = coef X with coef = -(w gamma), -(w gamma)^* or w; conjugations as signs
        const float ca = kind == 4 ? 0.f : -1.f, cw = kind == 4 ? 1.f : 0.f;
        const float cb_ = kind == 4 ? 0.f : (kind == 1 ? 1.f : -1.f);
        const float xs = kind == 2 ? -1.f : 1.f, ys = kind >= 3 ? -1.f : 1.f;
        const float fz1 = (float)z1;
        // TMEM lane quarter and column part this warp reads; the accumulator row it holds
        constexpr int kParts = kConvWarps / 4;
        const int quarter = warp & 3, part = warp >> 2;
        const int row = quarter * 32 + lane;
        const int rt = row / nb2, ri = row % nb2;
        const int ncol = a.npad / kParts, colb = part * ncol;  // ncol: a multiple of 8
        // the columns of this row's diagonal block inside this warp's part
        const int qlo = rt < ng ? max(0, rt * nb2 - colb) : 0;
        const int qhi = rt < ng ? min(ncol, rt * nb2 + nb2 - colb) : 0;

        // adds chain c's accumulator to dq (every element has one writer: its row's thread) and
        // hands the accumulator back to the MMA warp; 16 columns at a time, loads before stores
        auto flush = [&](int c, bool go) -> bool {
            if (go) go = wait_or_abort(smem_u32(&accfull[c & 1]), (c >> 1) & 1, &abort_flag, a.err);
            if (!conv_all(go)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((c & 1) * kTmemCols + colb);
            for (int q0 = 0; q0 < ncol; q0 += 8) {
                uint32_t v[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                               "=r"(v[6]), "=r"(v[7])
                             : "r"(base + (uint32_t)q0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float* d = dq + (colb + q0) * nb2 + ri;  // column colb + q0 + j at d[j * nb2]
                float o[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = (q0 + j >= qlo && q0 + j < qhi) ? d[j * nb2] : 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (q0 + j >= qlo && q0 + j < qhi) d[j * nb2] = o[j] + __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&accempty[c & 1]));
            return true;
        };

        int flushed = 0;
        bool good = true;
        for (int s = 0; s < ntiles; ++s) {
            const int slot = s % kRaw, st = s % kStages;
            if (good) good = wait_or_abort(smem_u32(&rawfull[slot]), (s / kRaw) & 1, &abort_flag, a.err);
            if (good && s >= kStages)
                good = wait_or_abort(smem_u32(&opempty[st]), ((s / kStages) - 1) & 1, &abort_flag, a.err);
            // one outcome per warp: a lane that saw the abort flag before the barrier completed
            // must not leave its warp split at the __syncwarp below
            good = __all_sync(0xffffffffu, good);
            if (good) {
                // ---- convert: L = coef X (conj), R = Y (conj), split hi/lo into the operand layout
                const float2* rx = reinterpret_cast<const float2*>(raw + slot * R.slot_bytes);
                const float2* ry = reinterpret_cast<const float2*>(raw + slot * R.slot_bytes + R.box_bytes);
                const float4* rc = reinterpret_cast<const float4*>(raw + slot * R.slot_bytes + 2 * R.box_bytes);
                unsigned char* sbase = ops + st * L::STAGE_BYTES;
                const int kend = c1 - (c0 + s * KT);  // centres of this stage inside the slice
#pragma unroll
                for (int q = 0; q < kItems; ++q) {
                    if (i_k[q] >= KT) continue;
                    float xr[PK], xi[PK], yr[PK], yi[PK];
#pragma unroll
                    for (int p = 0; p < PK; ++p) {
                        const int k = i_k[q] + p;
                        const float4 cf = rc[k];
                        float2 X = rx[i_xo[q] + p * nbp], Y = ry[i_yo[q] + p * nbp];
                        const bool use = k < kend && cf.w == fz1;
                        const float cr = ca * cf.x + cw * cf.z, ci = cb_ * cf.y;
                        X.y *= xs;
                        const float lx = cr * X.x - ci * X.y, ly = cr * X.y + ci * X.x;
                        xr[p] = use ? lx : 0.f;
                        xi[p] = use ? ly : 0.f;
                        yr[p] = use ? Y.x : 0.f;
                        yi[p] = use ? ys * Y.y : 0.f;
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
                    *reinterpret_cast<uint32_t*>(sbase + 0 * L::OP_BYTES + i_ore[q]) = h[0];
                    *reinterpret_cast<uint32_t*>(sbase + 1 * L::OP_BYTES + i_ore[q]) = l[0];
                    *reinterpret_cast<uint32_t*>(sbase + 0 * L::OP_BYTES + i_oim[q]) = h[1];
                    *reinterpret_cast<uint32_t*>(sbase + 1 * L::OP_BYTES + i_oim[q]) = l[1];
                    *reinterpret_cast<uint32_t*>(sbase + 2 * L::OP_BYTES + i_ore[q]) = h[2];
                    *reinterpret_cast<uint32_t*>(sbase + 3 * L::OP_BYTES + i_ore[q]) = l[2];
                    *reinterpret_cast<uint32_t*>(sbase + 2 * L::OP_BYTES + i_oim[q]) = h[3];
                    *reinterpret_cast<uint32_t*>(sbase + 3 * L::OP_BYTES + i_oim[q]) = l[3];
                }
                // make the generic-proxy stores visible to the tensor core; hand over the stage
                // and give the raw slot back to the TMA warp
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&opfull[st]));
                    mbar_arrive(smem_u32(&rawempty[slot]));
                }
            }
            // flush the previous chain once the next one is two tiles in (its MMAs are done by
            // then); all converter warps take part, so an abort ends the loop for all of them
            if (s % kFlush == 1 && s > kFlush) {
                good = flush(flushed, good);
                if (!good) break;
                ++flushed;
            }
        }
        // the remaining chains
        good = conv_all(good);
        while (good && flushed < nchains) {
            good = flush(flushed, true);
            ++flushed;
        }
    }

    __syncthreads();
    const bool ok = !abort_flag;
    if (!ok) {
        // a wait gave up: wait (bounded) for the copies still in flight and for the MMA warp's
        // last commit, which tracks all its MMAs, before the shared and tensor memory are freed
        if (warp == kConvWarps && lane == 0)
            for (int i = 0; i < kRaw; ++i) {
                const int s = last_tma - 1 - i;  // the last copy issued into each slot
                if (s >= 0) mbar_wait(smem_u32(&rawfull[s % kRaw]), (s / kRaw) & 1, a.err);
            }
        if (warp == kConvWarps + 1 && lane == 0 && last_mma > 0)
            mbar_wait(smem_u32(&opempty[(last_mma - 1) % kStages]), ((last_mma - 1) / kStages) & 1, a.err);
        __syncthreads();
    }
    // the complex block sums, in FP64: (Re L Re R - Im L Im R, Re L Im R + Im L Re R)
    for (int it = tid; it < ng * nbb; it += kThreads) {
        const int t = it / nbb, o = it % nbb, b1 = o / nb, b2 = o % nb;
        double re = 0.0, im = 0.0;
        if (ok) {
            const float* Dre = dq + (t * nb2 + b2) * nb2;       // column Re R(b2)
            const float* Dim = dq + (t * nb2 + nb + b2) * nb2;  // column Im R(b2)
            re = (double)Dre[b1] - (double)Dim[nb + b1];
            im = (double)Dim[b1] + (double)Dre[nb + b1];
        }
        double* dst = A.partial + 2 * (((size_t)sl * a.groups + (gbase + t)) * nbb + o);
        dst[0] = re;
        dst[1] = im;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols));
    }
}

// per-centre coefficients in centre order for the coefficient boxes: (w gamma_1, w gamma_2, w, zbin)
__global__ void centre_coef_kernel(int n, const int32_t* __restrict__ centre_idx, const Pay<float>* __restrict__ pay,
                                   const uint8_t* __restrict__ zs, float4* __restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int d = centre_idx[c];
        const Pay<float> p = pay[d];
        out[c] = make_float4(p.a, p.b, p.w, (float)(zs ? (int)zs[d] : 0));
    }
}

// slices of the centre axis: fill the resident CTA slots in whole waves, at least 8 stages
// of centres per slice, at most 64 slices
static int pick_slices(int tiles, int slots, int64_t n_centres, int kt)
{
    const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(64, n_centres / (8 * kt)));
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

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// FP32 tensor of rank 2 to 4 (dims innermost first, strides in bytes of dims 1..), boxes as given
static bool encode(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                   const uint32_t* box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class SP>
static cudaError_t launch_tc(TcArgs a, float4* coef, int n_sm, int* splits_out, bool plan_only, cudaStream_t st)
{
    const ContractArgs<float>& c = a.c;
    const size_t smem = smem_bytes<SP>(SP::KT, c.nb, a.nbp, a.gt);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_attr(contract_tc_kernel<SP>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = occupancy(&per_sm, contract_tc_kernel<SP>, kThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, 512 / (2 * kTmemCols)));
    const int tiles = c.nz * c.nz * c.nz * (4 * a.ta + a.tw);
    const int slices = a.fixed_slices > 0 ? (int)std::min<int64_t>(a.fixed_slices, std::max<int64_t>(1, c.n_centres))
                                          : pick_slices(tiles, per_sm * n_sm, c.n_centres, SP::KT);
    *splits_out = slices;
    if (plan_only) return cudaSuccess;
    if (slices != c.splits) return cudaErrorInvalidValue;  // partial buffer sized for another plan

    // tensor maps: order-major moments [orders][n_centres][nz][nbp] complex as FP32 (innermost first)
    const uint64_t nbp = (uint64_t)a.nbp, nz = (uint64_t)c.nz, nc = (uint64_t)c.n_centres;
    const uint32_t box[4] = {(uint32_t)(2 * nbp), 1u, (uint32_t)SP::KT, (uint32_t)a.gt};
    const uint64_t strides[3] = {nbp * 8, nz * nbp * 8, nc * nz * nbp * 8};
    CUtensorMap mg, mw, mc;
    {
        const uint64_t d[4] = {2 * nbp, nz, nc, (uint64_t)(2 * c.n_max + 3)};
        if (!encode(&mg, c.G, 4, d, strides, box)) return cudaErrorInvalidValue;
    }
    {
        const uint64_t d[4] = {2 * nbp, nz, nc, (uint64_t)(2 * c.n_max + 1)};
        if (!encode(&mw, c.W, 4, d, strides, box)) return cudaErrorInvalidValue;
    }
    {
        const uint64_t d[2] = {4, nc}, s[1] = {16};
        const uint32_t b2[2] = {4, (uint32_t)SP::KT};
        if (!encode(&mc, coef, 2, d, s, b2)) return cudaErrorInvalidValue;
    }
    centre_coef_kernel<<<(unsigned)std::min<int64_t>((nc + 255) / 256, 4 * n_sm), 256, 0, st>>>(
        c.n_centres, c.centre_idx, c.pay, c.zs, coef);
    contract_tc_kernel<SP><<<dim3(tiles, slices), kThreads, smem, st>>>(mg, mw, mc, a);
    return cudaGetLastError();
}

}  // namespace tc

cudaError_t launch_contract_tc(const ContractArgs<float>& c, bool tf32, int n_sm, float4* coef,
                               unsigned long long* err, int* splits, bool plan_only, int fixed_slices,
                               int skip_copies, cudaStream_t st)
{
    tc::TcArgs a;
    a.fixed_slices = fixed_slices;
    a.skip_copies = skip_copies;
    a.c = c;
    a.groups = c.nz * c.nz * c.nz * groups_per_zt(c.n_max);
    a.gt = std::min(tc::kMaxGroups, tc::kM / (2 * c.nb));
    if (a.gt < 1) return cudaErrorInvalidValue;
    a.npad = ((a.gt * 2 * c.nb + 31) / 32) * 32;
    a.nbp = nb_pad(c.nb);
    a.ta = (c.n_max + 1 + a.gt - 1) / a.gt;
    a.tw = (2 * c.n_max + 1 + a.gt - 1) / a.gt;
    a.err = err;
    return tf32 ? tc::launch_tc<tc::Tf32Split>(a, coef, n_sm, splits, plan_only, st)
                : tc::launch_tc<tc::Bf16Split>(a, coef, n_sm, splits, plan_only, st);
}

}  // namespace mp3
