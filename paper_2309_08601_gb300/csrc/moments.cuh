// Stage (a): radially binned harmonic moments of every centre galaxy's neighbours,
// G_m(i,b,Z) = sum_k w_k gamma_c,k e^{i m varphi_ik} and W_m(i,b,Z) = sum_k w_k e^{i m varphi_ik}
// (paper Sec. 3.1, Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization).
//
// Warp-specialised pipeline, one CTA per centre at a time (persistent over centres):
//  * the catalog is cell-sorted by (zbin, cell row, cell column), so the neighbours of a centre
//    that can fall in radial bin b are a short list of contiguous index ranges, one or two per
//    cell row crossed by the annulus [e_b, e_{b+1});
//  * the ranges of a bin are concatenated into one flat candidate stream (prefix sums of their
//    lengths) that is split evenly between NS producer warps; each streams its share with
//    coalesced loads of positions and payload records, several batches of 32 in flight (all
//    loads of a step are issued before any is used), test membership exactly on
//    the integer squared separation, and compact members (ballot + popc) into their own region
//    of one of two shared-memory chunks. A member stores z = (dx + i dy)/r, its powers
//    z^2..z^P, and w gamma_1, w gamma_2, w;
//  * P consumer warps split the moment orders by residue: consumer p owns m = p, p + P, ... so
//    all consumers do the same work. Each walks every member of a chunk, starts from z^p,
//    multiplies by z^P (complex recurrence in registers) and accumulates
//    A_m = sum w gamma_1 z^m, B_m = sum w gamma_2 z^m (m <= n_max + 3) and W_m = sum w z^m
//    (m <= 2 n_max) in registers;
//  * chunks are handed over through mbarriers (full / empty, double-buffered) whose waits are
//    bounded by a clock budget; a wait that runs out sets an abort flag that every other wait
//    also honours, and the kernel reports it instead of hanging;
//  * a chunk header carries (centre, Z, bin, flags); on the last chunk of a bin the consumers
//    reduce-scatter their per-lane sums across the warp and write G_m = A_m + i B_m,
//    G_{-m} = A_m^* + i B_m^* and W_m.
// The fixed range-to-producer assignment and per-producer regions make the summation order,
// and hence the result, reproducible run to run.
#pragma once

#include "common.cuh"

// Pipeline parameters (compile-time; the defaults are the tuned values).
#ifndef MP3_MOM_NS
#define MP3_MOM_NS 2  // producer warps
#endif
#ifndef MP3_MOM_UNR
#define MP3_MOM_UNR 4  // candidate batches of 32 a producer loads before using any
#endif
#ifndef MP3_MOM_CHUNK_F32
#define MP3_MOM_CHUNK_F32 512  // members per chunk buffer (FP32)
#endif
#ifndef MP3_MOM_MINB_F32
#define MP3_MOM_MINB_F32 3  // CTAs per SM the FP32 register budget is sized for
#endif
#ifndef MP3_MOM_WAIT_NS
#define MP3_MOM_WAIT_NS 0  // suspend-time hint (ns) of the producers' waits for a free buffer
#endif
#ifndef MP3_MOM_CWAIT_NS
#define MP3_MOM_CWAIT_NS 0  // suspend-time hint (ns) of the consumers' waits for a full buffer
#endif

namespace mp3 {

template <typename T>
struct MomTraits;
template <>
struct MomTraits<float> {
    static constexpr int kPerPart = 16;  // W orders per consumer warp (upper bound)
    static constexpr int kChunk = MP3_MOM_CHUNK_F32;  // members per chunk buffer
};
template <>
struct MomTraits<double> {
    static constexpr int kPerPart = 8;
    static constexpr int kChunk = 256;
};

template <typename T, int NMAX>
struct MomPlan {
    static constexpr int NM = 2 * NMAX + 1;
    static constexpr int P0 = (NM + MomTraits<T>::kPerPart - 1) / MomTraits<T>::kPerPart;
    static constexpr int P = P0 > 8 ? 8 : P0;  // consumer warps
    static constexpr int NS = sizeof(T) == 4 ? MP3_MOM_NS : 2;  // producer warps
    static constexpr int NT = 32 * (P + NS);
    static constexpr int CH = MomTraits<T>::kChunk;
    static constexpr int RC = CH / NS;  // producer region
    static constexpr int UNR = MP3_MOM_UNR;  // candidate batches of 32 in flight per producer
    static_assert(RC >= 32 * UNR, "region smaller than one producer step");
    static constexpr int NWM = (2 * NMAX) / P + 1;      // W orders of consumer 0
    static constexpr int NABM = (NMAX + 3) / P + 1;     // A, B orders of consumer 0
    static constexpr int NA = 4 * NABM + 2 * NWM;       // scalar accumulators
    static constexpr int NAP = (NA + 31) / 32 * 32;     // padded for the reduce-scatter
    // CTAs per SM the register budget is sized for
    static constexpr int MINB_R = 65536 / (NT * 96) > 0 ? 65536 / (NT * 96) : 1;
    static constexpr int MINB = sizeof(T) == 4 ? (MP3_MOM_MINB_F32 < MINB_R ? MP3_MOM_MINB_F32 : MINB_R) : 1;
};

template <typename T, int P, int CH>
struct MomSmem {
    cx<T> zp[2][P][CH];  // z^1 .. z^P of each member
    T a[2][CH], b[2][CH], w[2][CH];
    int cnt[2][8];   // members in each producer region
    int hdr[2][4];   // centre row, Z, bin, flags (1: last chunk of the bin, 2: last chunk)
    int2 seg[2 * kMaxRows];  // (first sorted index, count) of the current bin's ranges
    int pre[2 * kMaxRows + 1];  // exclusive prefix sums of the range lengths
    int wtot[8];                // per-producer-warp partial sums of the prefix scan
    long long e2q[kMaxBins + 1];
    unsigned long long full[2], empty[2];  // mbarriers
    int abort;
};

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, int parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try_wait_hint(unsigned long long* bar, int parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete. Gives up after ~2^31 SM clocks or when
// another wait of the CTA already gave up; then records the failure and returns false.
template <int HINT_NS>
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, int parity, volatile int* abort,
                                          unsigned long long* err)
{
    const long long t0 = clock64();
    while (!(HINT_NS > 0 ? mbar_try_wait_hint(bar, parity, HINT_NS) : mbar_try_wait(bar, parity))) {
        if (*abort) return false;
        if (clock64() - t0 > (1LL << 31)) {
            *abort = 1;
            atomicOr(err, 1ULL);
            return false;
        }
    }
    return true;
}

// barrier among the producer warps only (named barrier 1), optionally AND-reducing a predicate
template <int N>
__device__ __forceinline__ void producer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ bool producer_sync_and(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(N)
        : "memory");
    return r != 0;
}

template <typename T>
__device__ __forceinline__ cx<T> unit_vector(int dx, int dy, long long r2);

template <>
__device__ __forceinline__ cx<float> unit_vector<float>(int dx, int dy, long long r2)
{
    // |dx|, |dy| < 2^24 are exact in FP32; r^2 here only normalises z (the bin test used the
    // exact integer r2)
    (void)r2;
    const float fdx = (float)dx, fdy = (float)dy;
    const float rf = fdx * fdx + fdy * fdy;
    float inv = rsqrtf(rf);
    inv = inv * (1.5f - 0.5f * rf * inv * inv);  // one Newton step
    return {(float)dx * inv, (float)dy * inv};
}

template <>
__device__ __forceinline__ cx<double> unit_vector<double>(int dx, int dy, long long r2)
{
    const double inv = 1.0 / sqrt((double)r2);
    return {(double)dx * inv, (double)dy * inv};
}

// Reduce-scatter of N (multiple of 32) per-lane values over the warp: afterwards lane l holds
// the warp sums of indices [l*N/32, (l+1)*N/32) in v[0 .. N/32).
template <typename T, int N>
__device__ __forceinline__ void warp_reduce_scatter(T (&v)[N], int lane)
{
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 16 >> lvl;
        const int n = N >> lvl, half = n >> 1;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            if (i < half) {
                const T send = up ? v[i] : v[i + half];
                const T keep = up ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
}

// ------------------------------------------------------------------ producer

template <typename T, int NMAX>
__device__ __forceinline__ void moments_producer(const MomentArgs<T>& A,
                                                 MomSmem<T, MomPlan<T, NMAX>::P, MomPlan<T, NMAX>::CH>& s)
{
    using PL = MomPlan<T, NMAX>;
    constexpr int P = PL::P, NS = PL::NS, RC = PL::RC, UNR = PL::UNR;
    constexpr int NPT = 32 * NS;
    constexpr unsigned FULL = 0xffffffffu;
    const int q = (threadIdx.x >> 5) - P;  // producer index
    const int lane = threadIdx.x & 31, ptid = threadIdx.x - 32 * P;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nb = A.nb, nz = A.nz;
    const float S = (float)A.g.side;
    const float iS = 1.0f / S;
    volatile int* abort = &s.abort;
    int pb = 0;
    int ph_e[2] = {0, 0};
    bool used[2] = {false, false};

    for (int c = blockIdx.x; c < A.n_centres; c += gridDim.x) {
        const int ci = A.centre_idx[c];
        const int2 pc = A.pos[ci];
        const float fx = (float)((long long)pc.x - A.g.x0);
        const float fy = (float)((long long)pc.y - A.g.y0);
        const bool last_centre = c + (int)gridDim.x >= A.n_centres;
        for (int z = 0; z < nz; ++z) {
            for (int b = 0; b < nb; ++b) {
                const long long lo = s.e2q[b], hi = s.e2q[b + 1];
                const float Ro = sqrtf((float)hi) * 1.000001f + 4.0f;
                const float Ri = fmaxf(sqrtf((float)lo) * 0.999999f - 4.0f, 0.0f);
                int iy0 = (int)floorf((fy - Ro) * iS - 0.001f);
                int iy1 = (int)floorf((fy + Ro) * iS + 0.001f);
                iy0 = max(iy0, 0);
                iy1 = min(iy1, A.g.ncy - 1);
                int nrows = iy1 - iy0 + 1;
                nrows = nrows < 0 ? 0 : (nrows > kMaxRows ? kMaxRows : nrows);
                producer_sync<NPT>();  // the previous bin's ranges are no longer read
                for (int r = ptid; r < nrows; r += NPT) {
                    const int iy = iy0 + r;
                    const float ylo = (float)iy * S, yhi = ylo + S;
                    const float dymin = fmaxf(0.0f, fmaxf(ylo - fy, fy - yhi));
                    const float dymax = fmaxf(fabsf(fy - ylo), fabsf(fy - yhi));
                    int2 s0 = make_int2(0, 0), s1 = make_int2(0, 0);
                    const float ho2 = Ro * Ro - dymin * dymin + 1e-6f * Ro * Ro;
                    if (ho2 > 0.0f) {
                        const float hx = sqrtf(ho2);
                        const int ix0 = max((int)floorf((fx - hx) * iS - 0.001f), 0);
                        const int ix1 = min((int)floorf((fx + hx) * iS + 0.001f), A.g.ncx - 1);
                        if (ix0 <= ix1) {
                            int h0 = 1, h1 = 0;
                            const float hi2 = Ri * Ri - dymax * dymax - 1e-6f * Ri * Ri;
                            if (hi2 > 0.0f) {
                                const float hin = sqrtf(hi2) - 2.0f;
                                if (hin > 0.0f) {
                                    h0 = (int)ceilf((fx - hin) * iS + 0.001f);
                                    h1 = (int)floorf((fx + hin) * iS - 0.001f) - 1;
                                }
                            }
                            const int* cs = A.cell_start + (size_t)z * A.g.ncells + (size_t)iy * A.g.ncx;
                            if (h0 <= h1 && h0 <= ix1 && h1 >= ix0) {
                                const int l1 = min(h0 - 1, ix1);
                                if (l1 >= ix0) s0 = make_int2(cs[ix0], cs[l1 + 1] - cs[ix0]);
                                const int r0 = max(h1 + 1, ix0);
                                if (r0 <= ix1) s1 = make_int2(cs[r0], cs[ix1 + 1] - cs[r0]);
                            } else {
                                s0 = make_int2(cs[ix0], cs[ix1 + 1] - cs[ix0]);
                            }
                        }
                    }
                    s.seg[2 * r] = s0;
                    s.seg[2 * r + 1] = s1;
                }
                producer_sync<NPT>();
                const int n_seg = 2 * nrows;
                // ---- prefix sums of the range lengths: the ranges form one flat candidate
                //      stream, split evenly between the producer warps
                {
                    const int blk = (n_seg + NPT - 1) / NPT;
                    const int k0 = ptid * blk, k1 = min(k0 + blk, n_seg);
                    int loc = 0;
                    for (int k = k0; k < k1; ++k) loc += s.seg[k].y;
                    int incl = loc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (lane == 31) s.wtot[q] = incl;
                    producer_sync<NPT>();
                    int run = incl - loc, tot = 0;
                    for (int w = 0; w < NS; ++w) {
                        if (w < q) run += s.wtot[w];
                        tot += s.wtot[w];
                    }
                    for (int k = k0; k < k1; ++k) {
                        s.pre[k] = run;
                        run += s.seg[k].y;
                    }
                    if (ptid == 0) s.pre[n_seg] = tot;
                }
                producer_sync<NPT>();
                const int total = s.pre[n_seg];
                const int tq0 = (int)((long long)total * q / NS), tq1 = (int)((long long)total * (q + 1) / NS);
                // each lane walks the ranges: ks = range holding flat candidate t
                int tb = tq0;  // first flat candidate of the next step
                int ks = 0;
                {
                    int lo_k = 0, hi_k = n_seg;  // largest k with pre[k] <= tq0 + lane
                    const int t = tq0 + lane;
                    while (hi_k - lo_k > 1) {
                        const int mid = (lo_k + hi_k) >> 1;
                        if (s.pre[mid] <= t) lo_k = mid; else hi_k = mid;
                    }
                    ks = lo_k;
                }
                bool done = tb >= tq1;
                while (true) {
                    if (used[pb] && !*abort) {
                        mbar_wait<MP3_MOM_WAIT_NS>(&s.empty[pb], ph_e[pb], abort, A.pairs + 1);
                        ph_e[pb] ^= 1;
                    }
                    used[pb] = true;
                    int mycnt = 0;
                    const int base = q * RC;
                    while (!done && !*abort) {
                        if (mycnt > RC - 32 * UNR) break;
                        // UNR batches of 32 flat candidates, all loads issued before any use
                        int2 pp[UNR];
                        Pay<T> py[UNR];
                        bool ok[UNR];
#pragma unroll
                        for (int u = 0; u < UNR; ++u) {
                            const int t = tb + u * 32 + lane;
                            ok[u] = t < tq1;
                            while (ks + 1 < n_seg && s.pre[ks + 1] <= t) ++ks;
                            const int j = s.seg[ks].x + (t - s.pre[ks]);
                            if (ok[u]) {
                                pp[u] = A.pos[j];
                                py[u] = A.pay[j];
                            } else {
                                pp[u] = pc;
                                py[u] = Pay<T>{T(0), T(0), T(0), T(0)};
                            }
                        }
#pragma unroll
                        for (int u = 0; u < UNR; ++u) {
                            const int dx = pp[u].x - pc.x, dy = pp[u].y - pc.y;
                            const long long r2 = (long long)dx * dx + (long long)dy * dy;
                            const bool in = ok[u] && (r2 >= lo) && (r2 < hi);
                            const unsigned m = __ballot_sync(FULL, in);
                            if (in) {
                                const int slot = base + mycnt + __popc(m & lt_mask);
                                const cx<T> zu = unit_vector<T>(dx, dy, r2);
                                cx<T> zz = zu;
                                s.zp[pb][0][slot] = zu;
#pragma unroll
                                for (int k = 1; k < P; ++k) {
                                    zz = cmul(zz, zu);
                                    s.zp[pb][k][slot] = zz;
                                }
                                s.a[pb][slot] = py[u].a;
                                s.b[pb][slot] = py[u].b;
                                s.w[pb][slot] = py[u].w;
                            }
                            mycnt += __popc(m);
                        }
                        tb += 32 * UNR;
                        if (tb >= tq1) done = true;
                    }
                    if (*abort) done = true;
                    if (lane == 0) s.cnt[pb][q] = mycnt;
                    const bool all_done = producer_sync_and<NPT>(done);
                    if (ptid == 0) {
                        s.hdr[pb][0] = c;
                        s.hdr[pb][1] = z;
                        s.hdr[pb][2] = b;
                        s.hdr[pb][3] = (all_done ? 1 : 0) |
                                       ((all_done && last_centre && z == nz - 1 && b == nb - 1) ? 2 : 0);
                    }
                    mbar_arrive(&s.full[pb]);
                    pb ^= 1;
                    if (all_done) break;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ consumer

template <typename T, int NMAX>
__device__ __forceinline__ void moments_consumer(const MomentArgs<T>& A,
                                                 MomSmem<T, MomPlan<T, NMAX>::P, MomPlan<T, NMAX>::CH>& s,
                                                 T* stage)
{
    using PL = MomPlan<T, NMAX>;
    constexpr int P = PL::P, NS = PL::NS, RC = PL::RC;
    constexpr int NWM = PL::NWM, NABM = PL::NABM, NAP = PL::NAP;
    const int part = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const int MG = 2 * n_max + 3, MW = 2 * n_max + 1;
    // the last order slot of this consumer may fall outside the order range
    const bool lastW = part + (NWM - 1) * P <= 2 * NMAX;
    const bool lastAB = part + (NABM - 1) * P <= NMAX + 3;
    const int zsel = part > 0 ? part - 1 : 0;
    volatile int* abort = &s.abort;
    unsigned long long my_pairs = 0;

    T acc[NAP];
#pragma unroll
    for (int i = 0; i < NAP; ++i) acc[i] = T(0);

    int cb = 0;
    int ph_f[2] = {0, 0};
    while (true) {
        if (!mbar_wait<MP3_MOM_CWAIT_NS>(&s.full[cb], ph_f[cb], abort, A.pairs + 1)) break;
        ph_f[cb] ^= 1;
        const int c = s.hdr[cb][0], z = s.hdr[cb][1], b = s.hdr[cb][2], fl = s.hdr[cb][3];
#pragma unroll 1
        for (int qq = 0; qq < NS; ++qq) {
            const int cnt = s.cnt[cb][qq];
            my_pairs += (unsigned long long)cnt;
            const int e0 = qq * RC;
            for (int e = e0 + lane; e < e0 + cnt; e += 32) {
                const cx<T> zP = s.zp[cb][P - 1][e];
                cx<T> zq = s.zp[cb][zsel][e];
                if (part == 0) zq = cx<T>{T(1), T(0)};
                const T av = s.a[cb][e], bv = s.b[cb][e], wv = s.w[cb][e];
#pragma unroll
                for (int j = 0; j < NWM; ++j) {
                    if (j < NABM) {
                        if (j < NABM - 1 || lastAB) {
                            acc[4 * j + 0] += av * zq.x;
                            acc[4 * j + 1] += av * zq.y;
                            acc[4 * j + 2] += bv * zq.x;
                            acc[4 * j + 3] += bv * zq.y;
                        }
                    }
                    if (j < NWM - 1 || lastW) {
                        acc[4 * NABM + 2 * j + 0] += wv * zq.x;
                        acc[4 * NABM + 2 * j + 1] += wv * zq.y;
                    }
                    if (j + 1 < NWM) zq = cmul(zq, zP);
                }
            }
        }
        mbar_arrive(&s.empty[cb]);
        cb ^= 1;
        if (fl & 1) {
            // ---- end of (centre, Z, bin): reduce over the warp and write G, W
            warp_reduce_scatter<T, NAP>(acc, lane);
            constexpr int PER = NAP / 32;
            T* st = stage + part * NAP;
#pragma unroll
            for (int i = 0; i < PER; ++i) st[lane * PER + i] = acc[i];
            __syncwarp();
            const size_t row = ((size_t)c * nz + z) * nb + b;
            cx<T>* Gp = A.G + row * MG;
            cx<T>* Wp = A.W + row * MW;
            if (lane < NWM) {
                const int j = lane, m = part + j * P;
                if (m <= 2 * n_max) Wp[m] = cx<T>{st[4 * NABM + 2 * j], st[4 * NABM + 2 * j + 1]};
                if (j < NABM) {
                    const T ax = st[4 * j], ay = st[4 * j + 1], bx = st[4 * j + 2], by = st[4 * j + 3];
                    if (m <= n_max - 1) Gp[m + n_max + 3] = cx<T>{ax - by, ay + bx};
                    if (m >= 1 && m <= n_max + 3) Gp[n_max + 3 - m] = cx<T>{ax + by, bx - ay};
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < NAP; ++i) acc[i] = T(0);
        }
        if (fl & 2) break;
    }
    if (lane == 0 && my_pairs && part == 0) atomicAdd(A.pairs, my_pairs);
}

template <typename T, int NMAX>
__global__ void __launch_bounds__(MomPlan<T, NMAX>::NT, MomPlan<T, NMAX>::MINB) moments_kernel(const MomentArgs<T> A)
{
    using PL = MomPlan<T, NMAX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& s = *reinterpret_cast<MomSmem<T, PL::P, PL::CH>*>(smem_raw);
    T* stage = reinterpret_cast<T*>(smem_raw + sizeof(MomSmem<T, PL::P, PL::CH>));
    for (int i = threadIdx.x; i <= A.nb; i += blockDim.x) s.e2q[i] = A.e2q[i];
    if (threadIdx.x == 0) {
        mbar_init(&s.full[0], 32 * PL::NS);
        mbar_init(&s.full[1], 32 * PL::NS);
        mbar_init(&s.empty[0], 32 * PL::P);
        mbar_init(&s.empty[1], 32 * PL::P);
        s.abort = 0;
    }
    __syncthreads();
    if ((int)(threadIdx.x >> 5) < PL::P)
        moments_consumer<T, NMAX>(A, s, stage);
    else
        moments_producer<T, NMAX>(A, s);
}

template <typename T, int NMAX>
cudaError_t launch_moments_nmax(const MomentArgs<T>& a, int n_sm, cudaStream_t st)
{
    using PL = MomPlan<T, NMAX>;
    const size_t smem = sizeof(MomSmem<T, PL::P, PL::CH>) + sizeof(T) * PL::P * PL::NAP;
    cudaError_t e = cudaFuncSetAttribute(moments_kernel<T, NMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, moments_kernel<T, NMAX>, PL::NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)n_sm * per_sm;
    if (grid > a.n_centres) grid = a.n_centres;
    if (grid < 1) return cudaSuccess;
    moments_kernel<T, NMAX><<<(unsigned)grid, PL::NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments_dispatch(const MomentArgs<T>& a, int n_sm, cudaStream_t st)
{
    // the smallest compiled order set that covers n_max (extra orders are computed, not written)
    if (a.n_max <= 4) return launch_moments_nmax<T, 4>(a, n_sm, st);
    if (a.n_max <= 10) return launch_moments_nmax<T, 10>(a, n_sm, st);
    if (a.n_max <= 20) return launch_moments_nmax<T, 20>(a, n_sm, st);
    if (a.n_max <= 30) return launch_moments_nmax<T, 30>(a, n_sm, st);
    if (a.n_max <= 40) return launch_moments_nmax<T, 40>(a, n_sm, st);
    if (a.n_max <= 50) return launch_moments_nmax<T, 50>(a, n_sm, st);
    return cudaErrorInvalidValue;
}

}  // namespace mp3
