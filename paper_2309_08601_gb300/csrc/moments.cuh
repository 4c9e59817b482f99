// Stage (a): radially binned harmonic moments of every centre galaxy's neighbours,
// G_m(i,b,Z) = sum_k w_k gamma_c,k e^{i m varphi_ik} and W_m(i,b,Z) = sum_k w_k e^{i m varphi_ik}
// (paper Sec. 3.1, Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization).
//
// One CTA of P warps works on one centre at a time (persistent over centres).
//  * The catalog is cell-sorted by (zbin, cell row, cell column), so the neighbours of a centre
//    that can fall in radial bin b are a short list of contiguous index ranges, one or two per
//    cell row crossed by the annulus [e_b, e_{b+1}). The ranges are concatenated into one flat
//    candidate stream (prefix sums of their lengths) and split evenly between the warps.
//  * The bin is processed in rounds. Produce: each warp tests SCR candidates of its share,
//    exactly on the integer squared separation, and compacts the members (ballot + popc) into
//    its region of a shared-memory chunk, storing z = (dx + i dy)/r, its powers z^2..z^P, the
//    pair (w gamma_1, w gamma_2) as one 8-byte record (one shared load per member where two
//    4-byte loads cost 2.6 % of the kernel's time) and w. The candidates' positions and
//    payloads were copied into shared memory by cp.async one round earlier, so this phase does
//    not wait on memory.
//    Consume: warp p owns the orders m = p, p + P, p + 2P, ... (all warps do the same work),
//    walks every member of the chunk, steps through its orders with the three-term recurrence
//    c_{j+1} = 2 cos(P phi) c_j - c_{j-1} and accumulates A_m = sum w gamma_1 z^m,
//    B_m = sum w gamma_2 z^m (m <= n_max + 3) and W_m = sum w z^m (m <= 2 n_max) in registers;
//    in FP32 the real and imaginary parts of each update go through one packed two-lane FMA
//    (one instruction per order for the recurrence, and one each for A, B and W). Two CTA barriers separate the phases; the next round's
//    candidate copies are issued between them, so they land while the warps consume.
//  * At the end of a bin each warp reduce-scatters its per-lane sums across the warp and writes
//    G_m = A_m + i B_m, G_{-m} = A_m^* + i B_m^* and W_m of its orders.
// The fixed split of the candidate stream and the per-warp regions make the summation order,
// and hence the result, reproducible run to run.
#pragma once

#include "common.cuh"

// Tiling parameters (compile-time; the defaults are the tuned values).
// At n_max <= 30 (four warps) the FP32 kernel then holds 4 CTAs per SM: 128 registers per
// thread and 57 KB of shared memory per CTA (with kMaxRows = 480).
#ifndef MP3_MOM_SCR_F32
#define MP3_MOM_SCR_F32 160  // candidates per warp and round (FP32, <= 4 warps)
#endif
#ifndef MP3_MOM_SCR_F32_WIDE
#define MP3_MOM_SCR_F32_WIDE 96  // the same for n_max >= 32 (six or more warps per CTA)
#endif
#ifndef MP3_MOM_FFMA2
#define MP3_MOM_FFMA2 1  // FP32 sums through packed two-lane FMAs (n_max >= 32)
#endif
#ifndef MP3_MOM_MINB_F32
#define MP3_MOM_MINB_F32 4  // CTAs per SM the FP32 register budget is sized for (<= 4 warps)
#endif
#ifndef MP3_MOM_MINB_F32_WIDE
#define MP3_MOM_MINB_F32_WIDE 3  // the same for n_max >= 32 (six or more warps per CTA)
#endif

namespace mp3 {

template <typename T>
struct MomTraits;
template <>
struct MomTraits<float> {
    static constexpr int kPerPart = 16;  // W orders per warp (upper bound)
    static constexpr int kScr = MP3_MOM_SCR_F32;
};
template <>
struct MomTraits<double> {
    static constexpr int kPerPart = 8;
    static constexpr int kScr = 96;
};

template <typename T, int NMAX>
struct MomPlan {
    static constexpr int NM = 2 * NMAX + 1;
    static constexpr int P0 = (NM + MomTraits<T>::kPerPart - 1) / MomTraits<T>::kPerPart;
    static constexpr int P = P0 > 8 ? 8 : P0;  // warps = order residue classes
    static constexpr int NT = 32 * P;
    static constexpr bool WIDE = P > 4;
    static constexpr int SCR = sizeof(T) == 4 && WIDE ? MP3_MOM_SCR_F32_WIDE : MomTraits<T>::kScr;  // per warp and round
    static_assert(SCR % 32 == 0, "whole batches");
    static constexpr int CH = P * SCR;                // chunk capacity (members)
    static constexpr int NWM = (2 * NMAX) / P + 1;   // W orders of warp 0
    static constexpr int NABM = (NMAX + 3) / P + 1;  // A, B orders of warp 0
    static constexpr int NA = 4 * NABM + 2 * NWM;    // scalar accumulators
    static constexpr int NAP = (NA + 31) / 32 * 32;  // padded for the reduce-scatter
    static constexpr int MINB_R = 65536 / (NT * 112) > 0 ? 65536 / (NT * 112) : 1;
    static constexpr int MINB_F = WIDE ? MP3_MOM_MINB_F32_WIDE : MP3_MOM_MINB_F32;
    static constexpr int MINB = sizeof(T) == 4 ? (MINB_F < MINB_R ? MINB_F : MINB_R) : 1;
    // packed FP32 FMAs: measured faster with six or more warps per CTA (fewer CTAs per SM, the
    // FMA pipe the limit while consuming) and 2.5 % slower with four (issue slots to spare)
    static constexpr bool PACKED = sizeof(T) == 4 && WIDE && MP3_MOM_FFMA2 != 0;

};

template <typename T, int P, int SCR>
struct MomSmem {
    cx<T> zp[P][P * SCR];     // z^1 .. z^P of each member
    cx<T> ab[P * SCR];        // (w gamma_1, w gamma_2) of each member
    T w[P * SCR];
    int2 spos[P][SCR];        // staged candidate positions (cp.async, one round ahead)
    Pay<T> spay[P][SCR];      // staged candidate payloads
    int2 seg[2 * kMaxRows];   // (first sorted index, count) of the current bin's ranges
    int pre[2 * kMaxRows + 1];  // exclusive prefix sums of the range lengths
    long long e2q[kMaxBins + 1];
    int cnt[8];   // members in each warp's region this round
    int wtot[8];  // per-warp partial sums of the prefix scan
    int claim;    // the CTA's next centre from the work queue
};

template <typename T, int NMAX>
using MomSmemOf = MomSmem<T, MomPlan<T, NMAX>::P, MomPlan<T, NMAX>::SCR>;

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ cx<float> lds_cx(uint32_t a, float)
{
    cx<float> v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ cx<double> lds_cx(uint32_t a, double)
{
    cx<double> v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_r(uint32_t a, float)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_r(uint32_t a, double)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

// asynchronous global -> shared copies, completion tracked per thread (commit / wait groups)
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void stage_pay(Pay<T>* dst, const Pay<T>* src);
template <>
__device__ __forceinline__ void stage_pay<float>(Pay<float>* dst, const Pay<float>* src)
{
    cp_async16(dst, src);
}
template <>
__device__ __forceinline__ void stage_pay<double>(Pay<double>* dst, const Pay<double>* src)
{
    cp_async16(dst, src);
    cp_async16(reinterpret_cast<char*>(dst) + 16, reinterpret_cast<const char*>(src) + 16);
}

template <typename T>
__device__ __forceinline__ cx<T> unit_vector(int dx, int dy);

template <>
__device__ __forceinline__ cx<float> unit_vector<float>(int dx, int dy)
{
    // |dx|, |dy| < 2^24 are exact in FP32; r^2 here only normalises z (the bin test uses the
    // exact integer r^2)
    const float fdx = (float)dx, fdy = (float)dy;
    const float rf = fdx * fdx + fdy * fdy;
    float inv = rsqrtf(rf);
    inv = inv * (1.5f - 0.5f * rf * inv * inv);  // one Newton step
    return {fdx * inv, fdy * inv};
}

template <>
__device__ __forceinline__ cx<double> unit_vector<double>(int dx, int dy)
{
    const double inv = 1.0 / sqrt((double)dx * dx + (double)dy * dy);
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

// ------------------------------------------------------------------ per-lane accumulators
//
// A warp's sums of one (centre, z-bin, radial bin): A_m, B_m for its orders m = p + jP <= n_max + 3
// and W_m for m = p + jP <= 2 n_max, each complex. MomAcc<T>::add takes one member and runs the
// order recurrence c_{j+1} = kappa c_j - c_{j-1} (kappa = 2 cos(P phi)) over the warp's orders.
// flatten() writes them as NAP scalars, in the order the reduce-scatter expects
// (A_j.re, A_j.im, B_j.re, B_j.im for j < NABM, then W_j.re, W_j.im).
template <typename T, int NABM, int NWM, bool PACKED>
struct MomAcc {
    cx<T> a[NABM], b[NABM], w[NWM];

    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int j = 0; j < NABM; ++j) a[j] = b[j] = cx<T>{T(0), T(0)};
#pragma unroll
        for (int j = 0; j < NWM; ++j) w[j] = cx<T>{T(0), T(0)};
    }

    __device__ __forceinline__ void add(T av, T bv, T wv, T kappa, cx<T> c0, cx<T> c1, bool lastAB, bool lastW)
    {
#pragma unroll
        for (int j = 0; j < NWM; ++j) {
            if (j < NABM && (j < NABM - 1 || lastAB)) {
                a[j].x += av * c0.x;
                a[j].y += av * c0.y;
                b[j].x += bv * c0.x;
                b[j].y += bv * c0.y;
            }
            if (j < NWM - 1 || lastW) {
                w[j].x += wv * c0.x;
                w[j].y += wv * c0.y;
            }
            if (j + 1 < NWM) {
                const cx<T> c2{kappa * c1.x - c0.x, kappa * c1.y - c0.y};
                c0 = c1;
                c1 = c2;
            }
        }
    }

    template <int NAP>
    __device__ __forceinline__ void flatten(T (&acc)[NAP]) const
    {
#pragma unroll
        for (int j = 0; j < NABM; ++j) {
            acc[4 * j + 0] = a[j].x;
            acc[4 * j + 1] = a[j].y;
            acc[4 * j + 2] = b[j].x;
            acc[4 * j + 3] = b[j].y;
        }
#pragma unroll
        for (int j = 0; j < NWM; ++j) {
            acc[4 * NABM + 2 * j] = w[j].x;
            acc[4 * NABM + 2 * j + 1] = w[j].y;
        }
#pragma unroll
        for (int i = 4 * NABM + 2 * NWM; i < NAP; ++i) acc[i] = T(0);
    }
};

// FP32: the real and imaginary parts of every sum and of the recurrence are updated together by
// one packed two-lane FMA (__ffma2_rn, sm_100 and later), which halves the FMA instructions the
// warp issues and leaves issue slots to the loads and the member loop. The recurrence's
// subtraction is folded into the signs: the loop carries v_j = s_j c_j with
// s_j = +1, +1, -1, -1, +1, +1, ... (period 4), for which v_{j+1} = (-1)^j kappa v_j + v_{j-1}
// needs no negated addend; the sums of order slot j then hold s_j times their value and are
// multiplied by s_j in flatten(). Negation is exact, so the results are bit-identical to the
// scalar form above.
template <int NABM, int NWM>
struct MomAcc<float, NABM, NWM, true> {
    float2 a[NABM], b[NABM], w[NWM];

    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int j = 0; j < NABM; ++j) a[j] = b[j] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < NWM; ++j) w[j] = make_float2(0.0f, 0.0f);
    }

    __device__ __forceinline__ void add(float av, float bv, float wv, float kappa, cx<float> c0, cx<float> c1,
                                        bool lastAB, bool lastW)
    {
        const float2 av2 = make_float2(av, av), bv2 = make_float2(bv, bv), wv2 = make_float2(wv, wv);
        const float2 kp = make_float2(kappa, kappa), km = make_float2(-kappa, -kappa);
        float2 v0 = make_float2(c0.x, c0.y), v1 = make_float2(c1.x, c1.y);
#pragma unroll
        for (int j = 0; j < NWM; ++j) {
            if (j < NABM && (j < NABM - 1 || lastAB)) {
                a[j] = __ffma2_rn(av2, v0, a[j]);
                b[j] = __ffma2_rn(bv2, v0, b[j]);
            }
            if (j < NWM - 1 || lastW) w[j] = __ffma2_rn(wv2, v0, w[j]);
            if (j + 1 < NWM) {
                const float2 v2 = __ffma2_rn((j & 1) ? kp : km, v1, v0);
                v0 = v1;
                v1 = v2;
            }
        }
    }

    template <int NAP>
    __device__ __forceinline__ void flatten(float (&acc)[NAP]) const
    {
#pragma unroll
        for (int j = 0; j < NABM; ++j) {
            const float sg = (j & 2) ? -1.0f : 1.0f;
            acc[4 * j + 0] = sg * a[j].x;
            acc[4 * j + 1] = sg * a[j].y;
            acc[4 * j + 2] = sg * b[j].x;
            acc[4 * j + 3] = sg * b[j].y;
        }
#pragma unroll
        for (int j = 0; j < NWM; ++j) {
            const float sg = (j & 2) ? -1.0f : 1.0f;
            acc[4 * NABM + 2 * j] = sg * w[j].x;
            acc[4 * NABM + 2 * j + 1] = sg * w[j].y;
        }
#pragma unroll
        for (int i = 4 * NABM + 2 * NWM; i < NAP; ++i) acc[i] = 0.0f;
    }
};

// ------------------------------------------------------------------ kernel

template <typename T, int NMAX>
__global__ void __launch_bounds__(MomPlan<T, NMAX>::NT, MomPlan<T, NMAX>::MINB) moments_kernel(const MomentArgs<T> A)
{
    using PL = MomPlan<T, NMAX>;
    constexpr int P = PL::P, NT = PL::NT, SCR = PL::SCR, CH = PL::CH;
    constexpr int NWM = PL::NWM, NABM = PL::NABM, NAP = PL::NAP;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& s = *reinterpret_cast<MomSmemOf<T, NMAX>*>(smem_raw);
    T* stage = reinterpret_cast<T*>(smem_raw + sizeof(MomSmemOf<T, NMAX>));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const size_t plane = (size_t)A.n_centres * nz * A.nbp;  // stride between order slots
    const float S = (float)A.g.side, iS = 1.0f / S;
    // the last order slot of this warp may fall outside the order range
    const bool lastW = warp + (NWM - 1) * P <= 2 * NMAX;
    const bool lastAB = warp + (NABM - 1) * P <= NMAX + 3;
    const int zsel = warp > 0 ? warp - 1 : 0;
    const uint32_t zp_base = smem_u32(&s.zp[0][0]);
    const uint32_t ab_base = smem_u32(&s.ab[0]), w_base = smem_u32(&s.w[0]);
    const uint32_t aP = zp_base + (uint32_t)((P - 1) * CH * sizeof(cx<T>));
    const uint32_t aq = zp_base + (uint32_t)(zsel * CH * sizeof(cx<T>));
    int2* my_pos = s.spos[warp];
    Pay<T>* my_pay = s.spay[warp];
    unsigned long long my_pairs = 0;

    for (int i = tid; i <= nb; i += NT) s.e2q[i] = A.e2q[i];
    __syncthreads();

    MomAcc<T, NABM, NWM, PL::PACKED> macc;
    // Centres come from a work queue: a CTA starts with centre blockIdx.x and then claims the next
    // unprocessed one (one atomic per centre), so CTAs whose centres have fewer neighbours (masked
    // regions, patch edges, sparse z-bins) take more of them and all finish together. A centre's
    // result does not depend on the CTA that computes it.
    for (int c = blockIdx.x; c < A.n_centres;) {
        const int2 pc = A.pos[A.centre_idx[c]];
        const float fx = (float)((long long)pc.x - A.g.x0);
        const float fy = (float)((long long)pc.y - A.g.y0);
        for (int z = 0; z < nz; ++z) {
            for (int b = 0; b < nb; ++b) {
                const long long lo = s.e2q[b], hi = s.e2q[b + 1];
                // ---- index ranges of the cell rows the annulus crosses (conservative)
                const float Ro = sqrtf((float)hi) * 1.000001f + 4.0f;
                const float Ri = fmaxf(sqrtf((float)lo) * 0.999999f - 4.0f, 0.0f);
                int iy0 = (int)floorf((fy - Ro) * iS - 0.001f);
                int iy1 = (int)floorf((fy + Ro) * iS + 0.001f);
                iy0 = max(iy0, 0);
                iy1 = min(iy1, A.g.ncy - 1);
                int nrows = iy1 - iy0 + 1;
                nrows = nrows < 0 ? 0 : (nrows > kMaxRows ? kMaxRows : nrows);
                for (int r = tid; r < nrows; r += NT) {
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
                __syncthreads();
                const int n_seg = 2 * nrows;
                // ---- prefix sums of the range lengths (one flat candidate stream)
                {
                    const int blk = (n_seg + NT - 1) / NT;
                    const int k0 = tid * blk, k1 = min(k0 + blk, n_seg);
                    int loc = 0;
                    for (int k = k0; k < k1; ++k) loc += s.seg[k].y;
                    int incl = loc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (lane == 31) s.wtot[warp] = incl;
                    __syncthreads();
                    int run = incl - loc, tot = 0;
                    for (int w2 = 0; w2 < P; ++w2) {
                        if (w2 < warp) run += s.wtot[w2];
                        tot += s.wtot[w2];
                    }
                    for (int k = k0; k < k1; ++k) {
                        s.pre[k] = run;
                        run += s.seg[k].y;
                    }
                    if (tid == 0) s.pre[n_seg] = tot;
                }
                __syncthreads();
                const int total = s.pre[n_seg];
                const int tq0 = (int)((long long)total * warp / P);
                const int tq1 = (int)((long long)total * (warp + 1) / P);
                int ks = 0;  // range holding this lane's next candidate
                {
                    int lk = 0, hk = n_seg;  // largest k with pre[k] <= tq0 + lane
                    const int t = tq0 + lane;
                    while (hk - lk > 1) {
                        const int mid = (lk + hk) >> 1;
                        if (s.pre[mid] <= t) lk = mid; else hk = mid;
                    }
                    ks = lk;
                }
                // copies the positions and payloads of candidates [tb, tb + SCR) of this warp
                auto stage_candidates = [&](int tb) {
#pragma unroll
                    for (int u = 0; u < SCR / 32; ++u) {
                        const int t = tb + u * 32 + lane;
                        if (t < tq1) {
                            while (ks + 1 < n_seg && s.pre[ks + 1] <= t) ++ks;
                            const int j = s.seg[ks].x + (t - s.pre[ks]);
                            cp_async8(&my_pos[u * 32 + lane], &A.pos[j]);
                            stage_pay<T>(&my_pay[u * 32 + lane], &A.pay[j]);
                        }
                    }
                    cp_async_commit();
                };
                int tb = tq0;
                stage_candidates(tb);
                macc.reset();

                while (true) {
                    // ---- produce: this warp's staged candidates -> members in its region
                    cp_async_wait_all();
                    int mycnt = 0;
                    const int base = warp * SCR;
#pragma unroll
                    for (int u = 0; u < SCR / 32; ++u) {
                        const bool ok = tb + u * 32 + lane < tq1;
                        const int2 pu = ok ? my_pos[u * 32 + lane] : pc;
                        const int dx = pu.x - pc.x, dy = pu.y - pc.y;
                        const long long r2 = (long long)dx * dx + (long long)dy * dy;
                        const bool in = ok && (r2 >= lo) && (r2 < hi);
                        const unsigned m = __ballot_sync(FULL, in);
                        const int slot = base + mycnt + __popc(m & lt_mask);
                        // computed by every lane (no divergence), stored by members only
                        const cx<T> zu = unit_vector<T>(dx, dy);
                        cx<T> zz = zu;
                        if (in) s.zp[0][slot] = zu;
#pragma unroll
                        for (int k = 1; k < P; ++k) {
                            zz = cmul(zz, zu);
                            if (in) s.zp[k][slot] = zz;
                        }
                        if (in) {
                            const Pay<T> py = my_pay[u * 32 + lane];
                            s.ab[slot] = cx<T>{py.a, py.b};
                            s.w[slot] = py.w;
                        }
                        mycnt += __popc(m);
                    }
                    if (lane == 0) s.cnt[warp] = mycnt;
                    tb += SCR;
                    const bool more = __syncthreads_or(tb < tq1) != 0;
                    // the staging area is free: fetch the next round while consuming this one
                    if (tb < tq1) stage_candidates(tb);

                    // ---- consume: this warp's orders over every member of the chunk
#pragma unroll 1
                    for (int w2 = 0; w2 < P; ++w2) {
                        const int cnt = s.cnt[w2];
                        my_pairs += (unsigned long long)cnt;
                        const int e0 = w2 * SCR;
                        // orders m_j = warp + j P. With |z| = 1, z^{m+P} + z^{m-P} =
                        // 2 cos(P phi) z^m, so c_{j+1} = kappa c_j - c_{j-1}, kappa = 2 Re(z^P),
                        // real and imaginary parts alike. The recurrence runs at most NWM - 2
                        // steps, so its rounding error stays within a few hundred ulp of the
                        // directly multiplied power.
                        for (int e = e0 + lane; e < e0 + cnt; e += 32) {
                            const cx<T> zP = lds_cx(aP + e * (uint32_t)sizeof(cx<T>), T(0));
                            const cx<T> zq = lds_cx(aq + e * (uint32_t)sizeof(cx<T>), T(0));
                            const cx<T> abv = lds_cx(ab_base + e * (uint32_t)sizeof(cx<T>), T(0));
                            const T wv = lds_r(w_base + e * (uint32_t)sizeof(T), T(0));
                            const T kappa = zP.x + zP.x;
                            const cx<T> c0 = warp == 0 ? cx<T>{T(1), T(0)} : zq;
                            const cx<T> c1 = warp == 0 ? zP : cmul(zq, zP);
                            macc.add(abv.x, abv.y, wv, kappa, c0, c1, lastAB, lastW);
                        }
                    }
                    __syncthreads();  // the chunk may be overwritten
                    if (!more) break;
                }

                // ---- reduce over the warp and write G, W of (centre, Z, bin)
                T acc[NAP];
                macc.flatten(acc);
                warp_reduce_scatter<T, NAP>(acc, lane);
                constexpr int PER = NAP / 32;
                T* st = stage + warp * NAP;
#pragma unroll
                for (int i = 0; i < PER; ++i) st[lane * PER + i] = acc[i];
                __syncwarp();
                const size_t row = ((size_t)c * nz + z) * A.nbp + b;
                cx<T>* Gp = A.G + row;  // order slot q at Gp[q * plane]
                cx<T>* Wp = A.W + row;
                if (lane < NWM) {
                    const int j = lane, m = warp + j * P;
                    if (m <= 2 * n_max) Wp[m * plane] = cx<T>{st[4 * NABM + 2 * j], st[4 * NABM + 2 * j + 1]};
                    if (j < NABM) {
                        const T ax = st[4 * j], ay = st[4 * j + 1], bx = st[4 * j + 2], by = st[4 * j + 3];
                        if (m <= n_max - 1) Gp[(m + n_max + 3) * plane] = cx<T>{ax - by, ay + bx};
                        if (m >= 1 && m <= n_max + 3) Gp[(n_max + 3 - m) * plane] = cx<T>{ax + by, bx - ay};
                    }
                }
                __syncwarp();
            }
        }
        if (tid == 0) s.claim = (int)min(atomicAdd(A.queue, 1ull) + gridDim.x, (unsigned long long)A.n_centres);
        __syncthreads();
        c = s.claim;
    }
    if (tid == 0 && my_pairs) atomicAdd(A.pairs, my_pairs);
}

template <typename T, int NMAX>
cudaError_t launch_moments_nmax(const MomentArgs<T>& a, int n_sm, cudaStream_t st)
{
    using PL = MomPlan<T, NMAX>;
    const size_t smem = sizeof(MomSmemOf<T, NMAX>) + sizeof(T) * PL::P * PL::NAP;
    cudaError_t e = set_smem_attr(moments_kernel<T, NMAX>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = occupancy(&per_sm, moments_kernel<T, NMAX>, PL::NT, smem);
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
