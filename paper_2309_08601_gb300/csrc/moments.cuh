// Stage (a): radially binned harmonic moments of every centre galaxy's neighbours,
// G_m(i,b,Z) = sum_k w_k gamma_c,k e^{i m varphi_ik} and W_m(i,b,Z) = sum_k w_k e^{i m varphi_ik}
// (paper Sec. 3.1, Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization).
//
// Design (one CTA works on one centre at a time; persistent over centres):
//  * the catalog is cell-sorted by (zbin, cell row, cell column), so the neighbours of a centre
//    that can fall in radial bin b are a short list of contiguous index ranges, one or two per
//    cell row crossed by the annulus [e_b, e_{b+1});
//  * warp w streams ranges w, w + P, w + 2P, ... with coalesced int2 position loads, tests
//    membership exactly on the integer squared separation, and compacts the members (ballot +
//    popc) into its own region of a shared-memory chunk. Each member stores z = (dx + i dy)/r,
//    its powers z^2..z^P, and w gamma_1, w gamma_2, w. The fixed range-to-warp assignment and
//    the per-warp regions make the summation order, and so the result, reproducible;
//  * the moment orders are split over the P warps of the CTA by residue: warp p owns
//    m = p, p + P, p + 2P, ... so every warp does the same work. It walks the whole chunk,
//    starting from z^p and multiplying by z^P (complex recurrence in registers), and keeps
//    A_m = sum w gamma_1 z^m, B_m = sum w gamma_2 z^m (m <= n_max + 3) and
//    W_m = sum w z^m (m <= 2 n_max) in registers for the current bin;
//  * at the end of a bin the per-lane sums are reduced across the warp and written as
//    G_m = A_m + i B_m (m >= 0) and G_{-m} = A_m^* + i B_m^*.
// A is kept separate from B because w gamma_c = w gamma_1 + i w gamma_2 gives both G_m and
// G_{-m} = (sum (w gamma_c)^* z^m)^* from the same two real-weighted sums.
#pragma once

#include "common.cuh"

namespace mp3 {

template <typename T>
struct MomTraits;
template <>
struct MomTraits<float> {
    static constexpr int kPerPart = 16;  // W orders per warp
    static constexpr int kChunk = 1024;  // members per shared chunk
};
template <>
struct MomTraits<double> {
    static constexpr int kPerPart = 8;
    static constexpr int kChunk = 512;
};

template <typename T, int NMAX>
struct MomPlan {
    static constexpr int NM = 2 * NMAX + 1;
    static constexpr int P0 = (NM + MomTraits<T>::kPerPart - 1) / MomTraits<T>::kPerPart;
    static constexpr int P = P0 > 8 ? 8 : P0;
    static constexpr int CH = MomTraits<T>::kChunk;
    static constexpr int NT = 32 * P;
    // CTAs per SM the register budget is sized for (FP32: 12 warps per SM)
    static constexpr int MINB = sizeof(T) == 4 ? (384 / NT > 1 ? 384 / NT : 1) : 1;
    static_assert(CH >= 64 * P, "chunk too small for the fill bound");
    __host__ __device__ static constexpr int nw(int part) { return (2 * NMAX - part) / P + 1; }
    __host__ __device__ static constexpr int nab(int part)
    {
        return part <= NMAX + 3 ? (NMAX + 3 - part) / P + 1 : 0;
    }
};

template <typename T, int P, int CH>
struct MomSmem {
    cx<T> zp[P][CH];  // z^1 .. z^P of each member
    T a[CH], b[CH], w[CH];
    int2 seg[2 * kMaxRows];  // (first sorted index, count)
    long long e2q[kMaxBins + 1];
    int exhausted;
    int cnt[8];  // members in each warp's region this round
};

// CTA barrier that may be reached from different code locations by different warps (each warp
// runs its own specialisation of the loop nest); the non-.aligned form allows that.
__device__ __forceinline__ void cta_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ cx<T> unit_vector(int dx, int dy, long long r2);

template <>
__device__ __forceinline__ cx<float> unit_vector<float>(int dx, int dy, long long r2)
{
    const float rf = (float)r2;
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

template <typename T, int NMAX, int PART>
__device__ __forceinline__ void moments_body(const MomentArgs<T>& A,
                                             MomSmem<T, MomPlan<T, NMAX>::P, MomPlan<T, NMAX>::CH>& s)
{
    using PL = MomPlan<T, NMAX>;
    constexpr int P = PL::P, CH = PL::CH, NT = PL::NT;
    constexpr int NW = PL::nw(PART);
    constexpr int NAB = PL::nab(PART);
    constexpr int NABR = NAB > 0 ? NAB : 1;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int RC = CH / P;  // region of each warp in the chunk
    static_assert(RC >= 64, "region too small");
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nb = A.nb, nz = A.nz, n_max = A.n_max;
    const int MG = 2 * n_max + 3, MW = 2 * n_max + 1;
    const float S = (float)A.g.side;
    unsigned long long my_pairs = 0;

    for (int c = blockIdx.x; c < A.n_centres; c += gridDim.x) {
        const int ci = A.centre_idx[c];
        const int2 pc = A.pos[ci];
        const float fx = (float)((long long)pc.x - A.g.x0);
        const float fy = (float)((long long)pc.y - A.g.y0);
        for (int z = 0; z < nz; ++z) {
            for (int b = 0; b < nb; ++b) {
                const long long lo = s.e2q[b], hi = s.e2q[b + 1];
                // ---- index ranges of the cell rows the annulus crosses (conservative)
                const float Ro = sqrtf((float)hi) * 1.000001f + 4.0f;
                const float Ri = fmaxf(sqrtf((float)lo) * 0.999999f - 4.0f, 0.0f);
                int iy0 = (int)floorf((fy - Ro) / S - 0.001f);
                int iy1 = (int)floorf((fy + Ro) / S + 0.001f);
                iy0 = max(iy0, 0);
                iy1 = min(iy1, A.g.ncy - 1);
                int nrows = iy1 - iy0 + 1;
                nrows = nrows < 0 ? 0 : (nrows > kMaxRows ? kMaxRows : nrows);
                if (tid == 0) s.exhausted = 0;
                for (int r = tid; r < nrows; r += NT) {
                    const int iy = iy0 + r;
                    const float ylo = (float)iy * S, yhi = ylo + S;
                    const float dymin = fmaxf(0.0f, fmaxf(ylo - fy, fy - yhi));
                    const float dymax = fmaxf(fabsf(fy - ylo), fabsf(fy - yhi));
                    int2 s0 = make_int2(0, 0), s1 = make_int2(0, 0);
                    const float ho2 = Ro * Ro - dymin * dymin + 1e-6f * Ro * Ro;
                    if (ho2 > 0.0f) {
                        const float hx = sqrtf(ho2);
                        const int ix0 = max((int)floorf((fx - hx) / S - 0.001f), 0);
                        const int ix1 = min((int)floorf((fx + hx) / S + 0.001f), A.g.ncx - 1);
                        if (ix0 <= ix1) {
                            int h0 = 1, h1 = 0;
                            const float hi2 = Ri * Ri - dymax * dymax - 1e-6f * Ri * Ri;
                            if (hi2 > 0.0f) {
                                const float hin = sqrtf(hi2) - 2.0f;
                                if (hin > 0.0f) {
                                    h0 = (int)ceilf((fx - hin) / S + 0.001f);
                                    h1 = (int)floorf((fx + hin) / S - 0.001f) - 1;
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
                cta_sync();
                const int n_seg = 2 * nrows;

                cx<T> Aa[NABR], Bb[NABR], Ww[NW];
#pragma unroll
                for (int j = 0; j < NABR; ++j) Aa[j] = Bb[j] = cx<T>{T(0), T(0)};
#pragma unroll
                for (int j = 0; j < NW; ++j) Ww[j] = cx<T>{T(0), T(0)};

                int kseg = PART, cur = 0, end = 0;
                bool have = false, done = false;
                while (true) {
                    // ---- scan: fill this warp's region until it may overflow or its ranges end
                    int mycnt = 0;
                    while (!done) {
                        if (!have) {
                            if (kseg >= n_seg) {
                                done = true;
                                if (lane == 0) atomicAdd(&s.exhausted, 1);
                                break;
                            }
                            const int2 sg = s.seg[kseg];
                            kseg += P;
                            cur = sg.x;
                            end = sg.x + sg.y;
                            have = cur < end;
                            continue;
                        }
                        if (mycnt > RC - 32) break;
                        const int j = cur + lane;
                        bool in = false;
                        int dx = 0, dy = 0;
                        long long r2 = 0;
                        if (j < end) {
                            const int2 p = A.pos[j];
                            dx = p.x - pc.x;
                            dy = p.y - pc.y;
                            r2 = (long long)dx * dx + (long long)dy * dy;
                            in = (r2 >= lo) && (r2 < hi);
                        }
                        const unsigned m = __ballot_sync(FULL, in);
                        if (in) {
                            const int slot = PART * RC + mycnt + __popc(m & lt_mask);
                            const cx<T> zu = unit_vector<T>(dx, dy, r2);
                            cx<T> zz = zu;
                            s.zp[0][slot] = zu;
#pragma unroll
                            for (int q = 1; q < P; ++q) {
                                zz = cmul(zz, zu);
                                s.zp[q][slot] = zz;
                            }
                            s.a[slot] = A.pa[j];
                            s.b[slot] = A.pb[j];
                            s.w[slot] = A.pw[j];
                        }
                        mycnt += __popc(m);
                        cur += 32;
                        if (cur >= end) have = false;
                    }
                    if (lane == 0) s.cnt[PART] = mycnt;
                    cta_sync();
                    const bool all_done = (s.exhausted == P);
                    // ---- accumulate this warp's orders over every region of the chunk
                    int n = 0;
#pragma unroll 1
                    for (int w = 0; w < P; ++w) {
                        const int cw = s.cnt[w];
                        n += cw;
                        for (int e = w * RC + lane; e < w * RC + cw; e += 32) {
                            const cx<T> zP = s.zp[P - 1][e];
                            cx<T> zq;
                            if constexpr (PART == 0) {
                                zq = cx<T>{T(1), T(0)};
                            } else {
                                zq = s.zp[PART - 1][e];
                            }
                            const T av = s.a[e], bv = s.b[e], wv = s.w[e];
#pragma unroll
                            for (int j = 0; j < NW; ++j) {
                                if (j < NAB) {
                                    Aa[j].x += av * zq.x;
                                    Aa[j].y += av * zq.y;
                                    Bb[j].x += bv * zq.x;
                                    Bb[j].y += bv * zq.y;
                                }
                                Ww[j].x += wv * zq.x;
                                Ww[j].y += wv * zq.y;
                                if (j + 1 < NW) zq = cmul(zq, zP);
                            }
                        }
                    }
                    if (tid == 0) my_pairs += (unsigned long long)n;
                    cta_sync();
                    if (all_done) break;
                }

                // ---- reduce over the warp and write G, W of (centre, Z, bin)
#pragma unroll
                for (int j = 0; j < NW; ++j) {
                    Ww[j].x = warp_sum(Ww[j].x);
                    Ww[j].y = warp_sum(Ww[j].y);
                    if (j < NAB) {
                        Aa[j].x = warp_sum(Aa[j].x);
                        Aa[j].y = warp_sum(Aa[j].y);
                        Bb[j].x = warp_sum(Bb[j].x);
                        Bb[j].y = warp_sum(Bb[j].y);
                    }
                }
                if (lane == 0) {
                    const size_t row = ((size_t)c * nz + z) * nb + b;
                    cx<T>* Gp = A.G + row * MG;
                    cx<T>* Wp = A.W + row * MW;
#pragma unroll
                    for (int j = 0; j < NW; ++j) {
                        const int m = PART + j * P;
                        if (m <= 2 * n_max) Wp[m] = Ww[j];
                        if (j < NAB) {
                            if (m <= n_max - 1)
                                Gp[m + n_max + 3] = cx<T>{Aa[j].x - Bb[j].y, Aa[j].y + Bb[j].x};
                            if (m >= 1 && m <= n_max + 3)
                                Gp[n_max + 3 - m] = cx<T>{Aa[j].x + Bb[j].y, Bb[j].x - Aa[j].y};
                        }
                    }
                }
            }
        }
    }
    if (tid == 0 && my_pairs) atomicAdd(A.pairs, my_pairs);
}

template <typename T, int NMAX>
__global__ void __launch_bounds__(MomPlan<T, NMAX>::NT, MomPlan<T, NMAX>::MINB) moments_kernel(const MomentArgs<T> A)
{
    using PL = MomPlan<T, NMAX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& s = *reinterpret_cast<MomSmem<T, PL::P, PL::CH>*>(smem_raw);
    for (int i = threadIdx.x; i <= A.nb; i += blockDim.x) s.e2q[i] = A.e2q[i];
    __syncthreads();
    const int part = threadIdx.x >> 5;
    // each warp runs the loop nest with its own compile-time order set; the loops are uniform
    // across the CTA, so every warp meets the same sequence of barriers
    switch (part) {
#define MP3_PART(q)                                          \
    case q:                                                  \
        if constexpr (q < PL::P) moments_body<T, NMAX, q>(A, s); \
        break;
        MP3_PART(0)
        MP3_PART(1)
        MP3_PART(2)
        MP3_PART(3)
        MP3_PART(4)
        MP3_PART(5)
        MP3_PART(6)
        MP3_PART(7)
#undef MP3_PART
        default:
            break;
    }
}

template <typename T, int NMAX>
cudaError_t launch_moments_nmax(const MomentArgs<T>& a, int n_sm, cudaStream_t st)
{
    using PL = MomPlan<T, NMAX>;
    const size_t smem = sizeof(MomSmem<T, PL::P, PL::CH>);
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
