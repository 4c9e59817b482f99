// Stage (b) on the 5th-generation tensor cores (tcgen05): the multipole components
// Upsilon_{mu,n}(b1,b2) and N_n(b1,b2) as real GEMMs over the centre-galaxy axis (paper
// Sec. 3.1, Eqs. Upsilon0_Derivation, Upsilon1-3, 3PCF_Normalization, tomoGn).
//
// A group g = (Z-triplet, component, order n) is the complex product sum_i L_i(b1) R_i(b2) with
// L = c_i X_i (c_i = -w gamma, -(w gamma)^*, or w) and R = Y_i. Written in reals with the Re and
// Im parts of a bin on neighbouring rows (columns), the rows of L times the columns of R give
// 2x2 blocks whose combination is the complex result. Components share moment rows: for one order
// n, the two left operands -w gamma G_{n-3} and -w gamma G_{-n-1}^* and the two right operands
// G_{-n-3} and G_{n-1}^* give Upsilon_0, Upsilon_3, Upsilon_2 and (transposed and conjugated)
// Upsilon_1 of the triplet with Z2 and Z3 exchanged, so one M = 128 tile of 4 n_bins rows and
// columns computes four components from four moment rows with no block wasted (n_bins <= 32).
// Tiles of N_n hold two orders (the two diagonal blocks are kept); with Z2 = Z3 their left and
// right operands are the same moment rows, copied once.
//
// Split precision: every operand value x is written as hi + lo with hi = round(x) and
// lo = round(x - hi) in BF16 (or TF32), and D += A_hi B_hi + A_hi B_lo + A_lo B_hi is
// accumulated in FP32 in tensor memory (the lo*lo term is below the rounding of the others).
// The tensor core's FP32 accumulation is not round-to-nearest: over thousands of centres its
// error grows with the number of accumulating MMAs (measured: 1e-4 relative after ~1700 BF16 or
// ~3400 TF32 MMAs, TF32 worse). So every kFlush stages the accumulator is read out (tcgen05.ld),
// combined into complex values and added to FP32 block sums in shared memory by the CUDA cores,
// and restarted: no chain is longer than 3 kFlush KT / KI MMAs.
//
// Pipeline per CTA (one tile, one slice of the centre axis), warp-specialised: one TMA warp copies
// the moment rows and coefficients of the next KT centres into a ring of raw slots; sixteen
// converter warps form c X and Y, split them and store them in the canonical no-swizzle K-major
// operand layout (8-row x 16-byte core matrices) of one of two stages; one MMA warp issues the
// three split products of a stage and commits them to the stage's barrier and, at the end of a
// chain, to the accumulator's; the converter warps flush a finished accumulator while the MMAs
// fill the other. Every wait on an mbarrier is bounded (about a second); a wait that gives up sets
// bit 2 of the error word and an abort flag that ends every role's loop, waits (bounded) for the
// copies and MMAs in flight and frees the tensor memory. The per-slice sums are written as FP64
// partials and summed in a fixed order by contract_reduce_kernel, so results are deterministic.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace mp3 {

namespace tc {

constexpr int kConvWarps = 16;                 // converter warps: four per TMEM lane quarter
constexpr int kThreads = (kConvWarps + 2) * 32;  // + one TMA warp + one MMA warp
constexpr int kM = 128;         // MMA rows (TMEM lanes)
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

// A tile of the contraction: up to two sides s, each with a left operand L_s = c X_s (X_s a moment
// row of z-bin Z2, conjugated or not, c the centre's coefficient) and a right operand R_s = Y_s
// (a moment row of z-bin Z3, conjugated or not). The MMA forms every product L_s R_t; the tile
// lists which blocks (s, t) are components and where they go.
//
// Paired tiles (4 n_bins <= 128), one per order n of Upsilon: with c = -(w gamma),
//   X_0 = G_{n-3},  Y_0 = G_{-n-3},  X_1 = G_{-n-1}^*,  Y_1 = G_{n-1}^*,
// so that (0,0) = Upsilon_0,n, (0,1) = Upsilon_3,n, (1,0) = Upsilon_2,n of the Z-triplet and
// (1,1)(b1, b2) = conj(Upsilon_1,n(b2, b1)) of the triplet with Z2 and Z3 exchanged (Eqs.
// Upsilon0_Derivation, Upsilon1-3): four components from four moment rows. N tiles hold two
// orders n, n+1 (c = w, X_s = W_{n+s}, Y_s = W_{n+s}^*), blocks (0,0) and (1,1) only.
// Single tiles (n_bins > 32): one component per tile.
struct TileSpec {
    int z1, z2, z3;
    int ns;              // sides with data
    int mapw;            // 0: G moments, 1: W moments
    int ox[2], oy[2];    // order slots of X_s and Y_s
    float xs[2], ys[2];  // +1, or -1 for the complex conjugate
    float cb, cw;        // c = -w gamma_1 + i cb w gamma_2 (cw = 0), or c = w (cw = 1)
    int nblk;
    int bl[4], br[4], bg[4], bt[4];  // block: left side, right side, group, 1 = transposed conjugate
};

__host__ __device__ inline int tiles_per_zt(int pair, int n_max)
{
    return pair ? 2 * (n_max + 1) : 4 * (n_max + 1) + 2 * n_max + 1;
}

__device__ void make_tile(TileSpec& t, int tile, int pair, int nz, int n_max)
{
    const int per = tiles_per_zt(pair, n_max);
    const int zt = tile / per, r = tile % per;
    t.z1 = zt / (nz * nz);
    t.z2 = (zt / nz) % nz;
    t.z3 = zt % nz;
    const int zsw = (t.z1 * nz + t.z3) * nz + t.z2;  // Z2 and Z3 exchanged
    const int gpz = groups_per_zt(n_max), offg = n_max + 3;
    auto gid = [&](int z, int kind, int n) { return z * gpz + (kind < 4 ? kind * (n_max + 1) : 4 * (n_max + 1)) + n; };
    auto side = [&](int s, int ox, float xs, int oy, float ys) {
        t.ox[s] = ox;
        t.xs[s] = xs;
        t.oy[s] = oy;
        t.ys[s] = ys;
    };
    auto block = [&](int i, int l, int rr, int g, int tr) {
        t.bl[i] = l;
        t.br[i] = rr;
        t.bg[i] = g;
        t.bt[i] = tr;
    };
    side(1, 0, 1.f, 0, 1.f);
    if (pair && r <= n_max) {
        const int n = r;
        t.ns = 2;
        t.mapw = 0;
        side(0, n - 3 + offg, 1.f, -n - 3 + offg, 1.f);
        side(1, -n - 1 + offg, -1.f, n - 1 + offg, -1.f);
        t.cb = -1.f, t.cw = 0.f;
        t.nblk = 4;
        block(0, 0, 0, gid(zt, 0, n), 0);
        block(1, 0, 1, gid(zt, 3, n), 0);
        block(2, 1, 0, gid(zt, 2, n), 0);
        block(3, 1, 1, gid(zsw, 1, n), 1);
    } else if (pair) {
        const int n0 = 2 * (r - n_max - 1);
        t.ns = min(2, 2 * n_max + 1 - n0);
        t.mapw = 1;
        t.cb = 0.f, t.cw = 1.f;
        t.nblk = t.ns;
        for (int s = 0; s < t.ns; ++s) {
            side(s, n0 + s, 1.f, n0 + s, -1.f);
            block(s, s, s, gid(zt, 4, n0 + s), 0);
        }
    } else {
        t.ns = 1;
        t.nblk = 1;
        t.cb = -1.f, t.cw = 0.f;
        const int kind = min(4, r / (n_max + 1)), n = kind < 4 ? r % (n_max + 1) : r - 4 * (n_max + 1);
        t.mapw = kind == 4;
        switch (kind) {
            case 0: side(0, n - 3 + offg, 1.f, -n - 3 + offg, 1.f); break;    // G_{n-3} G_{-n-3}
            case 1: side(0, n - 1 + offg, 1.f, -n - 1 + offg, 1.f); t.cb = 1.f; break;  // -(w gamma)^*
            case 2: side(0, -n - 1 + offg, -1.f, -n - 3 + offg, 1.f); break;  // G_{-n-1}^* G_{-n-3}
            case 3: side(0, n - 3 + offg, 1.f, n - 1 + offg, -1.f); break;    // G_{n-3} G_{n-1}^*
            default: side(0, n, 1.f, n, -1.f); t.cb = 0.f, t.cw = 1.f; break;  // W_n W_n^*
        }
        block(0, 0, 0, gid(zt, kind, n), 0);
    }
}

struct TcArgs {
    ContractArgs<float> c;
    int groups;        // nz^3 * groups_per_zt(n_max): index space of the partial sums
    int pair;          // 1: two sides per tile (4 nb <= 128 rows), 0: one side (2 nb <= 128)
    int npad;          // MMA N: 2 nb columns per side, rounded up to 32 (8 TMEM columns per part)
    int nbp;           // bins padded to even (the moment rows)
    int fixed_slices;  // > 0: this many centre slices instead of the automatic choice
    int skip_copies;   // test hook: issue no TMA copies, so every wait on them runs out
    unsigned long long* err;
};

// one raw slot: boxes X_0 [X_1] Y_0 [Y_1], each one order row [KT centres][nbp bins] complex,
// then the coefficients [KT]
struct RawLayout {
    int box_bytes, slot_bytes, sides;
    __host__ __device__ RawLayout(int kt, int nbp, int pair)
    {
        sides = pair ? 2 : 1;
        box_bytes = kt * nbp * 8;
        slot_bytes = ((2 * sides * box_bytes + kt * 16) + 127) / 128 * 128;
    }
};

// one operand stage: A_hi, A_lo, B_hi, B_lo, each 128 rows x KT centres in the canonical no-swizzle
// K-major layout: element (r, k) at ((r/8)*(KT/T) + k/T)*128 B + (r%8)*16 B + (k%T)*ES. Row
// 2b + side 2nb holds Re of bin b, the next row Im.
template <class SP>
struct Layout {
    static constexpr int T = 16 / SP::ES;                 // elements per 16-byte core row
    static constexpr int KT = SP::KT;
    static constexpr int SBO = (KT / T) * 128;            // bytes between 8-row core groups
    static constexpr int OP_BYTES = kM * KT * SP::ES;
    static constexpr int STAGE_BYTES = 4 * OP_BYTES;
    static constexpr int PK = 4 / SP::ES;                 // centres per 32-bit word
    static constexpr int KW = KT / PK;                    // 32-bit words along K per row
    static_assert(KW == 8, "a warp covers 4 bins x 8 words");
    __device__ static uint32_t word_off(int r, int kw)
    {
        // kw-th 32-bit word of row r: centres kw*PK .. kw*PK + PK - 1
        return (uint32_t)((r / 8) * SBO + (kw / 4) * 128 + (r % 8) * 16 + (kw % 4) * 4);
    }
};

constexpr int kRaw = 3;    // raw slots: the TMA copies run two stages ahead of the conversion
constexpr int kDqs = 129;  // floats between the columns of the block sums (rows 0..127, padded)

template <class SP>
static size_t smem_bytes(int kt, int nbp, int pair, int npad)
{
    const RawLayout R(kt, nbp, pair);
    return (size_t)kRaw * R.slot_bytes + kStages * (size_t)Layout<SP>::STAGE_BYTES +
           (size_t)(npad / 2) * kDqs * sizeof(float);
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

// Grid: x = tiles (TileSpec), y = slices of the centre axis. Warp roles: warps 0..kConvWarps-1
// convert raw moments into split operands and flush the accumulators; warp kConvWarps issues the
// TMA copies; warp kConvWarps+1 issues the MMAs. They synchronise only through mbarriers:
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
    __shared__ TileSpec ts;

    const ContractArgs<float>& A = a.c;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const int nbb = nb * nb, nb2 = 2 * nb, nbp = a.nbp;
    const RawLayout R(KT, nbp, a.pair);
    unsigned char* raw = smem;
    unsigned char* ops = smem + kRaw * R.slot_bytes;
    // FP32 block sums: column pair p (Re R, Im R of one bin) of row r at dq[p * kDqs + r]; even
    // rows hold the real part of the complex block element, odd rows the imaginary part
    float* dq = reinterpret_cast<float*>(ops + kStages * L::STAGE_BYTES);
    const int dq_floats = (a.npad / 2) * kDqs;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        make_tile(ts, blockIdx.x, a.pair, nz, n_max);
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
    // zero the operand stages (rows and columns outside the sides stay zero) and the block sums
    {
        uint4* z = reinterpret_cast<uint4*>(ops);
        const int n16 = (kStages * L::STAGE_BYTES + dq_floats * 4 + 15) / 16;
        for (int i = tid; i < n16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int ns = ts.ns, z1 = ts.z1;

    // slices of the centres of z-bin z1 (a contiguous range of the z-sorted centre list)
    const int sl = blockIdx.y, slices = gridDim.y;
    const int zc0 = A.zrange ? A.zrange[z1] : 0, zc1 = A.zrange ? A.zrange[z1 + 1] : A.n_centres;
    const int per = (zc1 - zc0 + slices - 1) / slices;
    const int c0 = min(zc1, zc0 + sl * per), c1 = min(zc1, c0 + per);
    const int ntiles = (c1 - c0 + KT - 1) / KT;
    const int nchains = (ntiles + kFlush - 1) / kFlush;
    // Y_s is the same row as X_s (same z-bin and order): one box serves both
    auto y_alias = [&](int s) { return ts.z2 == ts.z3 && ts.ox[s] == ts.oy[s]; };

    if (warp == kConvWarps) {
        // ================= TMA warp: copies of tile s into raw slot s % kRaw. Lanes 0..nbox-1
        // copy one moment row each and lane nbox the coefficients, all in one warp instruction
        const CUtensorMap* mapM = ts.mapw ? &mapW : &mapG;
        int nbox = 0, my_off = 0, my_z = 0, my_o = 0;
        for (int q = 0; q < ns; ++q) {
            if (lane == nbox) my_off = q * R.box_bytes, my_z = ts.z2, my_o = ts.ox[q];
            ++nbox;
            if (!y_alias(q)) {
                if (lane == nbox) my_off = (R.sides + q) * R.box_bytes, my_z = ts.z3, my_o = ts.oy[q];
                ++nbox;
            }
        }
        const bool coef_lane = lane == nbox, active = lane <= nbox;
        if (coef_lane) my_off = 2 * R.sides * R.box_bytes;
        const uint32_t tx_bytes = nbox * R.box_bytes + KT * 16;
        for (int s = 0; s < ntiles; ++s) {
            const int slot = s % kRaw;
            bool go = true;
            if (lane == 0 && s >= kRaw)
                go = wait_or_abort(smem_u32(&rawempty[slot]), ((s / kRaw) - 1) & 1, &abort_flag, a.err);
            if (!__shfl_sync(0xffffffffu, go ? 1 : 0, 0)) break;
            if (a.skip_copies) continue;
            const uint32_t dst = smem_u32(raw + slot * R.slot_bytes);
            const uint32_t bar = smem_u32(&rawfull[slot]);
            const int cb = c0 + s * KT;
            if (lane == 0) mbar_expect_tx(bar, tx_bytes);
            __syncwarp();
            if (active) {
                if (coef_lane)
                    tma_load_2d(dst + my_off, &mapC, 0, cb, bar);
                else
                    tma_load_4d(dst + my_off, mapM, 0, my_z, cb, my_o, bar);
            }
            if (lane == 0) last_tma = s + 1;
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
        // Warp w converts four bins of one side: bin 4 (w % nbq) + (lane / 4) % 4 of side
        // w / nbq, 32-bit word column 4 (lane / 16) + lane % 4 (PK centres). Each lane writes its
        // bin's Re row and Im row; the lanes of the upper half-warp write Im first, so every store
        // instruction covers 8 distinct rows of a core group x 4 words (no bank conflicts).
        // Conjugations are not applied here: a side with X conjugated stores c^* X = conj(c X^*)
        // (its Im row negated) and R is stored as Y; the flush applies both signs.
        const int nbq = (nb + 3) / 4;
        const int side = warp / nbq, b = 4 * (warp % nbq) + ((lane >> 2) & 3);
        const int ph = lane >> 4, kw = 4 * ph + (lane & 3);
        const bool item = side < ns && b < nb;
        const int sd = item ? side : 0;
        const int rre = sd * nb2 + 2 * b;
        const uint32_t o1 = L::word_off(rre + ph, kw), o2 = L::word_off(rre + 1 - ph, kw);
        const int k0 = kw * PK;
        const int xoff = sd * R.box_bytes, yoff = (y_alias(sd) ? sd : R.sides + sd) * R.box_bytes;
        // coefficients (-w gamma_1, -w gamma_2, w, zbin): c = -w gamma, or -(w gamma)^* (cb > 0),
        // or w (N tiles); cis: the sign of Im c', c' = c or c^*
        const bool wcoef = ts.cw != 0.f;
        const float cis = -ts.cb * ts.xs[sd];
        // TMEM lane quarter and column part this warp reads; the accumulator row it holds
        constexpr int kParts = kConvWarps / 4;
        const int quarter = warp & 3, part = warp >> 2;
        const int row = quarter * 32 + lane;
        const int ncol = a.npad / kParts, colb = part * ncol;  // ncol: a multiple of 8
        const float sx = ts.xs[min(row / nb2, 1)];

        // adds chain c's accumulator to dq and hands it back to the MMA warp. The lanes of the A
        // rows Re and Im of a bin are neighbours: with (e0, e1) = (A_re B_re, A_re B_im) and
        // (o0, o1) = (A_im B_re, A_im B_im), A_im = sx Im L and B_im = sy Im R, the even lane keeps
        // Re(L R) = e0 - sx sy o1, the odd one Im(L R) = sy e1 + sx o0; each dq element has one
        // writer
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
                const int cp0 = (colb + q0) >> 1;
                float* d = dq + cp0 * kDqs + row;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float sy = ts.ys[min((cp0 + j) / nb, 1)];
                    const float e = __uint_as_float(v[2 * j]);
                    const float t = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[2 * j + 1]), 1);
                    d[j * kDqs] += (lane & 1) ? sy * t + sx * e : e - sx * sy * t;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&accempty[c & 1]));
            return true;
        };

        // L' = c' X and R = Y of this lane's bin, split hi/lo and stored; RAG: the stage ends
        // inside the slice (centres k >= kend are zero); WC: real coefficient w
        auto convert = [&](const unsigned char* rs, unsigned char* sbase, int kend, auto rag_t, auto wc_t) {
            constexpr bool RAG = decltype(rag_t)::value, WC = decltype(wc_t)::value;
            const float2* rx = reinterpret_cast<const float2*>(rs + xoff);
            const float2* ry = reinterpret_cast<const float2*>(rs + yoff);
            const float4* rc = reinterpret_cast<const float4*>(rs + 2 * R.sides * R.box_bytes);
            float xr[PK], xi[PK], yr[PK], yi[PK];
#pragma unroll
            for (int p = 0; p < PK; ++p) {
                const int k = k0 + p;
                const float4 cf = rc[k];
                const float2 X = rx[k * nbp + b], Y = ry[k * nbp + b];
                float lx, ly;
                if constexpr (WC) {
                    lx = cf.z * X.x;
                    ly = cf.z * X.y;
                } else {
                    const float ci = cis * cf.y;
                    lx = cf.x * X.x - ci * X.y;
                    ly = cf.x * X.y + ci * X.x;
                }
                const bool use = !RAG || k < kend;
                xr[p] = use ? lx : 0.f;
                xi[p] = use ? ly : 0.f;
                yr[p] = use ? Y.x : 0.f;
                yi[p] = use ? Y.y : 0.f;
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
            // (first, second) row of this lane: (Re, Im), or (Im, Re) in the upper half-warp
            auto put = [&](int op, uint32_t re, uint32_t im) {
                *reinterpret_cast<uint32_t*>(sbase + op * L::OP_BYTES + o1) = ph ? im : re;
                *reinterpret_cast<uint32_t*>(sbase + op * L::OP_BYTES + o2) = ph ? re : im;
            };
            put(0, h[0], h[1]);
            put(1, l[0], l[1]);
            put(2, h[2], h[3]);
            put(3, l[2], l[3]);
        };

        int flushed = 0;
        bool good = true;
        for (int s = 0; s < ntiles; ++s) {
            const int slot = s % kRaw, st = s % kStages;
            // warp 0 waits for the stage's copies and operand buffer; the others wait for warp 0
            // at a named barrier, which also gives every converter thread the same outcome
            if (warp == 0 && good) good = wait_or_abort(smem_u32(&rawfull[slot]), (s / kRaw) & 1, &abort_flag, a.err);
            if (warp == 0 && good && s >= kStages)
                good = wait_or_abort(smem_u32(&opempty[st]), ((s / kStages) - 1) & 1, &abort_flag, a.err);
            good = conv_all(good);
            if (good) {
                const unsigned char* rs = raw + slot * R.slot_bytes;
                unsigned char* sbase = ops + st * L::STAGE_BYTES;
                const int kend = c1 - (c0 + s * KT);  // centres of this stage inside the slice
                if (item) {
                    if (kend >= KT) {
                        if (wcoef)
                            convert(rs, sbase, kend, std::false_type{}, std::true_type{});
                        else
                            convert(rs, sbase, kend, std::false_type{}, std::false_type{});
                    } else {
                        if (wcoef)
                            convert(rs, sbase, kend, std::true_type{}, std::true_type{});
                        else
                            convert(rs, sbase, kend, std::true_type{}, std::false_type{});
                    }
                }
                // make the generic-proxy stores visible to the tensor core; each warp then hands
                // over its part of the stage and of the raw slot (the barriers count the warps)
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
    // the tile's blocks in FP64: element (b1, b2) of block (l, r) is row 2 b1 + l 2nb (Re) and the
    // next row (Im) of column pair b2 + r nb; a transposed-conjugate block reads (b2, b1), -Im
    for (int it = tid; it < ts.nblk * nbb; it += kThreads) {
        const int k = it / nbb, o = it % nbb, b1 = o / nb, b2 = o % nb;
        const int tr = ts.bt[k];
        const int r0 = ts.bl[k] * nb2 + 2 * (tr ? b2 : b1), cp = ts.br[k] * nb + (tr ? b1 : b2);
        double re = 0.0, im = 0.0;
        if (ok) {
            re = (double)dq[cp * kDqs + r0];
            im = (double)dq[cp * kDqs + r0 + 1];
            if (tr) im = -im;
        }
        double* dst = A.partial + 2 * (((size_t)sl * a.groups + ts.bg[k]) * nbb + o);
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

// per-centre coefficients in centre order for the coefficient boxes: (-w gamma_1, -w gamma_2, w, zbin)
__global__ void centre_coef_kernel(int n, const int32_t* __restrict__ centre_idx, const Pay<float>* __restrict__ pay,
                                   const uint8_t* __restrict__ zs, float4* __restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int d = centre_idx[c];
        const Pay<float> p = pay[d];
        out[c] = make_float4(-p.a, -p.b, p.w, (float)(zs ? (int)zs[d] : 0));
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
    const size_t smem = smem_bytes<SP>(SP::KT, a.nbp, a.pair, a.npad);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_attr(contract_tc_kernel<SP>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = occupancy(&per_sm, contract_tc_kernel<SP>, kThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, 512 / (2 * kTmemCols)));
    const int tiles = c.nz * c.nz * c.nz * tiles_per_zt(a.pair, c.n_max);
    const int slices = a.fixed_slices > 0 ? (int)std::min<int64_t>(a.fixed_slices, std::max<int64_t>(1, c.n_centres))
                                          : pick_slices(tiles, per_sm * n_sm, c.n_centres, SP::KT);
    *splits_out = slices;
    if (plan_only) return cudaSuccess;
    if (slices != c.splits) return cudaErrorInvalidValue;  // partial buffer sized for another plan

    // tensor maps: order-major moments [orders][n_centres][nz][nbp] complex as FP32 (innermost first)
    const uint64_t nbp = (uint64_t)a.nbp, nz = (uint64_t)c.nz, nc = (uint64_t)c.n_centres;
    const uint32_t box[4] = {(uint32_t)(2 * nbp), 1u, (uint32_t)SP::KT, 1u};
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
    if (2 * c.nb > tc::kM) return cudaErrorInvalidValue;
    a.pair = 4 * c.nb <= tc::kM ? 1 : 0;
    a.npad = (((a.pair ? 2 : 1) * 2 * c.nb + 31) / 32) * 32;
    a.nbp = nb_pad(c.nb);
    a.err = err;
    return tf32 ? tc::launch_tc<tc::Tf32Split>(a, coef, n_sm, splits, plan_only, st)
                : tc::launch_tc<tc::Bf16Split>(a, coef, n_sm, splits, plan_only, st);
}

}  // namespace mp3
