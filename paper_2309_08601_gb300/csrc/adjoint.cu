// Adjoint (reverse mode) of stages (b) and (a): given dL/dUpsilon and dL/dN for a real loss L,
// the gradient with respect to every galaxy's w gamma and w (paper Sec. 3.1: Eqs.
// Upsilon0_Derivation, Upsilon1-3, 3PCF_Normalization, tomoGn for (b); the moment sums of
// Sec. 3.1 for (a)).
//
// Convention: for a complex quantity z, grad z = dL/dRe z + i dL/dIm z. For y = a z,
// grad z += conj(a) grad y; for y = a conj(z), grad z += a conj(grad y); for a real parameter t in
// y = t h, dL/dt += Re(conj(grad y) h).
//
// Stage (b), per group (Z-triplet, component, n) with y(b1, b2) = sum_i c_i X_i(b1) Y_i(b2):
//   grad X_i(b1) = conj(c_i) sum_b2 grad y(b1, b2) conj(Y_i(b2)),
//   grad Y_i(b2) = conj(c_i) sum_b1 grad y(b1, b2) conj(X_i(b1)),
//   grad c_i     = sum_b1 conj(X_i(b1)) sum_b2 grad y(b1, b2) conj(Y_i(b2)),
// with an extra conjugation where the moment enters conjugated. dL/dG and dL/dW are gathered per
// output moment element (each written once, no atomics): an element receives the X or Y role of
// at most eight (component, n) groups.
//
// Stage (a): G_m(i, b) = sum_k v_k e^{i m phi_ik} and W_m(i, b) = sum_k w_k e^{i m phi_ik}, so
//   grad v_k += sum_{i, m} grad G_m(i, b_ik) e^{-i m phi_ik},
//   dL/dw_k  += Re sum_{i, m} grad W_m(i, b_ik) e^{-i m phi_ik}.
// For each (centre, bin) the adjoint moments are the coefficients of a trigonometric polynomial
// evaluated at every neighbour's angle by Horner's rule (in u = e^{-i phi} for m >= 0 and in
// z = e^{i phi} for m < 0), one neighbour per lane, and added to the neighbour's gradient with
// atomics (the gradient is therefore not bit-reproducible). Neighbours are found per bin from
// the cell grid of the forward pass: for every cell row, the one or two runs of cells that meet
// the annulus.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace mp3 {

namespace adj {

template <typename T>
__device__ __forceinline__ cx<T> ld(const cx<T>* p, size_t i)
{
    return p[i];
}

__device__ __forceinline__ cx<double> ldd(const double* p, size_t i)
{
    return cx<double>{p[2 * i], p[2 * i + 1]};
}

template <typename T>
__device__ __forceinline__ cx<T> to_t(cx<double> v)
{
    return cx<T>{(T)v.x, (T)v.y};
}

template <typename T>
__device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b)
{
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
}

// ------------------------------------------------------------------ stage (b): dL/dG, dL/dW

constexpr int kTileC = 32;  // centres per block

// the gradient tables of AdjArgs (tabX transposed so that the X role reads consecutive bins)
template <typename T>
__global__ void grad_tables(const AdjArgs<T> a, int64_t n_ups_groups, int64_t total)
{
    const int nb = a.nb, nbb = nb * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i / nbb;
        const int o = (int)(i % nbb), b1 = o / nb, b2 = o % nb;
        const cx<double> v = g < n_ups_groups ? ldd(a.gups, i) : ldd(a.gnorm, i - n_ups_groups * nbb);
        a.tabY[i] = to_t<T>(v);
        a.tabX[g * nbb + (int64_t)b2 * nb + b1] = to_t<T>(v);
    }
}

// grid: x = centre tiles, y = output order slot (G slots 0..MG-1, then W slots); thread per
// (centre, z, bin) output element
template <typename T>
__global__ void __launch_bounds__(256) contract_adjoint_moments(const AdjArgs<T> a)
{
    const int nb = a.nb, nz = a.nz, nmax = a.n_max, nbp = nb_pad(nb);
    const int MG = 2 * nmax + 3, o = nmax + 3, NN = nmax + 1, NW = 2 * nmax + 1;
    const int q = blockIdx.y;
    const bool isG = q < MG;
    const int m = isG ? q - o : q - MG;
    const size_t plane = (size_t)a.n_centres * nz * nbp;
    for (int e = threadIdx.x; e < kTileC * nz * nb; e += blockDim.x) {
        const int b = e % nb, z = (e / nb) % nz;
        const int c = blockIdx.x * kTileC + e / (nb * nz);
        if (c >= a.n_centres) continue;
        const int d = a.centre_idx[c];
        const Pay<T> pv = a.pay[d];
        const int z1 = a.zs ? (int)a.zs[d] : 0;
        const cx<T> v{pv.a, pv.b};
        const cx<T> c0{-v.x, -v.y}, c1{-v.x, v.y};  // -v and -conj(v)
        const cx<T> cw{pv.w, T(0)};
        const size_t crow = (size_t)c * nz;
        // X role: output at b1 = b, partner Y at order slot qy of Z zo; returns
        // conj(coef) sum_b2 grad y(b, b2) conj(Y(b2)) (grad y from the transposed table: the
        // lanes, consecutive in b, read consecutive elements)
        const size_t nbb = (size_t)nb * nb, n_off = (size_t)nz * nz * nz * 4 * NN * nbb;
        auto roleX = [&](const cx<T>* M, size_t gbase, int zo, int qy, bool yconj, cx<T> coef) {
            cx<T> s{T(0), T(0)};
            const cx<T>* Y = M + (size_t)qy * plane + (crow + zo) * nbp;
            const cx<T>* gt = a.tabX + gbase + b;
            for (int b2 = 0; b2 < nb; ++b2) {
                cx<T> y = Y[b2];
                if (!yconj) y.y = -y.y;  // conj(Y) (conj(conj(G)) = G when Y enters conjugated)
                cfma(s, gt[(size_t)b2 * nb], y);
            }
            return cmul(s, cconj(coef));
        };
        // Y role: output at b2 = b, partner X at order slot qx of Z zo
        auto roleY = [&](const cx<T>* M, size_t gbase, int zo, int qx, bool xconj, cx<T> coef) {
            cx<T> s{T(0), T(0)};
            const cx<T>* X = M + (size_t)qx * plane + (crow + zo) * nbp;
            const cx<T>* gt = a.tabY + gbase + b;
            for (int b1 = 0; b1 < nb; ++b1) {
                cx<T> x = X[b1];
                if (!xconj) x.y = -x.y;
                cfma(s, gt[(size_t)b1 * nb], x);
            }
            return cmul(s, cconj(coef));
        };
        auto ub = [&](int zt, int kind, int n) { return ((((size_t)zt * 4 + kind) * NN + n) * nb) * nb; };
        cx<T> acc{T(0), T(0)};
        if (isG) {
            for (int zo = 0; zo < nz; ++zo) {
                const int ztX = (z1 * nz + z) * nz + zo;  // this element as X (Z2 = z), partner Z3 = zo
                const int ztY = (z1 * nz + zo) * nz + z;  // this element as Y (Z3 = z), partner Z2 = zo
                int n;
                // kind 0: G_{n-3}(b1) G_{-n-3}(b2), coef -v
                n = m + 3;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleX(a.G, ub(ztX, 0, n), zo, -n - 3 + o, false, c0));
                n = -m - 3;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleY(a.G, ub(ztY, 0, n), zo, n - 3 + o, false, c0));
                // kind 1: G_{n-1}(b1) G_{-n-1}(b2), coef -conj(v)
                n = m + 1;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleX(a.G, ub(ztX, 1, n), zo, -n - 1 + o, false, c1));
                n = -m - 1;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleY(a.G, ub(ztY, 1, n), zo, n - 1 + o, false, c1));
                // kind 2: conj(G_{-n-1}(b1)) G_{-n-3}(b2), coef -v
                n = -m - 1;
                if (n >= 0 && n <= nmax)
                    acc = cadd(acc, cconj(roleX(a.G, ub(ztX, 2, n), zo, -n - 3 + o, false, c0)));
                n = -m - 3;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleY(a.G, ub(ztY, 2, n), zo, -n - 1 + o, true, c0));
                // kind 3: G_{n-3}(b1) conj(G_{n-1}(b2)), coef -v
                n = m + 3;
                if (n >= 0 && n <= nmax) acc = cadd(acc, roleX(a.G, ub(ztX, 3, n), zo, n - 1 + o, true, c0));
                n = m + 1;
                if (n >= 0 && n <= nmax)
                    acc = cadd(acc, cconj(roleY(a.G, ub(ztY, 3, n), zo, n - 3 + o, false, c0)));
            }
            a.gG[(size_t)q * plane + (crow + z) * nbp + b] = acc;
        } else {
            const int n = m;
            for (int zo = 0; zo < nz; ++zo) {
                const int ztX = (z1 * nz + z) * nz + zo, ztY = (z1 * nz + zo) * nz + z;
                // N_n: w W_n(b1) conj(W_n(b2))
                const size_t nX = n_off + (((size_t)ztX * NW + n) * nb) * nb;
                const size_t nY = n_off + (((size_t)ztY * NW + n) * nb) * nb;
                acc = cadd(acc, roleX(a.W, nX, zo, n, true, cw));
                acc = cadd(acc, cconj(roleY(a.W, nY, zo, n, false, cw)));
            }
            a.gW[(size_t)n * plane + (crow + z) * nbp + b] = acc;
        }
    }
}

// grad of every centre's own coefficient: a warp per centre (kCoefCentres centres per warp), lanes
// over b1; per group the block stages the group's transposed dL/dy in shared memory (skipped when
// none of the block's centres is in the group's Z1) and each warp forms
// gc = sum_b1 conj(X(b1)) sum_b2 dL/dy(b1, b2) conj(Y(b2)) (partner rows read as warp broadcasts),
// then adds dL/dv (re, im) and dL/dw of the centre's sorted galaxy
constexpr int kCoefWarps = 8, kCoefCentres = 4;

template <typename T>
__global__ void __launch_bounds__(kCoefWarps * 32) contract_adjoint_coef(const AdjArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* gyT = reinterpret_cast<cx<T>*>(smem_raw);  // [nb][nb]: gyT[b2 * nb + b1]
    const int nb = a.nb, nz = a.nz, nmax = a.n_max, nbp = nb_pad(nb), nbb = nb * nb;
    const int o = nmax + 3, NN = nmax + 1, NW = 2 * nmax + 1;
    const int per_zt = groups_per_zt(nmax);
    const size_t plane = (size_t)a.n_centres * nz * nbp;
    const int64_t nU = (int64_t)nz * nz * nz * 4 * NN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cbase = (blockIdx.x * kCoefWarps + warp) * kCoefCentres;
    int dd[kCoefCentres], zc[kCoefCentres];
    cx<T> gv[kCoefCentres];
    T gw[kCoefCentres];
    unsigned zmask = 0;  // z-bins of this warp's centres
#pragma unroll
    for (int j = 0; j < kCoefCentres; ++j) {
        const int c = cbase + j;
        dd[j] = c < a.n_centres ? a.centre_idx[c] : -1;
        zc[j] = dd[j] >= 0 ? (a.zs ? (int)a.zs[dd[j]] : 0) : -1;
        if (zc[j] >= 0) zmask |= 1u << (zc[j] & 31);
        gv[j] = cx<T>{T(0), T(0)};
        gw[j] = T(0);
    }
    const int groups = nz * nz * nz * per_zt;
    for (int g = 0; g < groups; ++g) {
        const int zt = g / per_zt, loc = g % per_zt;
        const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
        if (!__syncthreads_or((zmask >> (z1 & 31)) & 1u)) continue;  // no centre of the block in Z1
        int kind, n;
        if (loc < 4 * NN) {
            kind = loc / NN;
            n = loc % NN;
        } else {
            kind = 4;
            n = loc - 4 * NN;
        }
        const int64_t tg = kind < 4 ? ((int64_t)zt * 4 + kind) * NN + n : nU + (int64_t)zt * NW + n;
        const cx<T>* src = a.tabX + tg * nbb;  // already transposed: [b2][b1]
        for (int i = threadIdx.x; i < nbb; i += blockDim.x) gyT[i] = src[i];
        __syncthreads();
        int qx, qy;
        bool xc = false, yc = false;
        switch (kind) {
            case 0: qx = n - 3 + o; qy = -n - 3 + o; break;
            case 1: qx = n - 1 + o; qy = -n - 1 + o; break;
            case 2: qx = -n - 1 + o; qy = -n - 3 + o; xc = true; break;
            case 3: qx = n - 3 + o; qy = n - 1 + o; yc = true; break;
            default: qx = n; qy = n; yc = true; break;
        }
        const cx<T>* M = kind < 4 ? a.G : a.W;
#pragma unroll
        for (int j = 0; j < kCoefCentres; ++j) {
            if (zc[j] != z1) continue;  // warp-uniform
            const int c = cbase + j;
            const cx<T>* X = M + (size_t)qx * plane + ((size_t)c * nz + z2) * nbp;
            const cx<T>* Y = M + (size_t)qy * plane + ((size_t)c * nz + z3) * nbp;
            cx<T> part{T(0), T(0)};
            for (int b1 = lane; b1 < nb; b1 += 32) {
                cx<T> sy{T(0), T(0)};
                for (int b2 = 0; b2 < nb; ++b2) {
                    cx<T> y = Y[b2];
                    if (!yc) y.y = -y.y;
                    cfma(sy, gyT[b2 * nb + b1], y);
                }
                cx<T> x = X[b1];
                if (!xc) x.y = -x.y;
                cfma(part, x, sy);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                part.x += __shfl_xor_sync(0xffffffffu, part.x, off);
                part.y += __shfl_xor_sync(0xffffffffu, part.y, off);
            }
            if (kind == 4) {
                gw[j] += part.x;  // c = w
            } else if (kind == 1) {
                gv[j].x -= part.x;  // c = -conj(v): grad v = -conj(grad c)
                gv[j].y += part.y;
            } else {
                gv[j].x -= part.x;  // c = -v
                gv[j].y -= part.y;
            }
        }
        __syncthreads();
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kCoefCentres; ++j)
            if (dd[j] >= 0) {
                a.gvw[4 * (size_t)dd[j]] += gv[j].x;
                a.gvw[4 * (size_t)dd[j] + 1] += gv[j].y;
                a.gvw[4 * (size_t)dd[j] + 2] += gw[j];
            }
    }
}

// ------------------------------------------------------------------ stage (a): pair loop

__device__ __forceinline__ long long isqrt_floor(long long v)
{
    if (v <= 0) return 0;
    long long r = (long long)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

__device__ __forceinline__ long long fdiv(long long a, long long b)
{
    const long long q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// adds (re grad v, im grad v, grad w) to a galaxy's 16-byte (FP32) or 32-byte (FP64) slot
__device__ __forceinline__ void atomic_add_vw(float* p, float vr, float vi, float w)
{
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(vr, vi, w, 0.0f));
}
__device__ __forceinline__ void atomic_add_vw(double* p, double vr, double vi, double w)
{
    atomicAdd(p, vr);
    atomicAdd(p + 1, vi);
    atomicAdd(p + 2, w);
}

template <typename T>
__device__ __forceinline__ cx<T> unit_dir(long long dx, long long dy);
template <>
__device__ __forceinline__ cx<float> unit_dir<float>(long long dx, long long dy)
{
    const float fx = (float)dx, fy = (float)dy;
    const float ir = rsqrtf(fx * fx + fy * fy);
    return {fx * ir, fy * ir};
}
template <>
__device__ __forceinline__ cx<double> unit_dir<double>(long long dx, long long dy)
{
    const double fx = (double)dx, fy = (double)dy;
    const double ir = 1.0 / sqrt(fx * fx + fy * fy);
    return {fx * ir, fy * ir};
}

constexpr int kPairWarps = 4;

// one Horner step p <- p x + c in four fused multiply-adds
template <typename T>
__device__ __forceinline__ cx<T> horner_step(cx<T> p, cx<T> x, cx<T> c)
{
    return {fma(p.x, x.x, fma(-p.y, x.y, c.x)), fma(p.x, x.y, fma(p.y, x.x, c.y))};
}

// Walks the candidates of redshift bin z around the centre (px, py): the warp goes row by row of
// the cell grid over the one or two runs of cells that meet the annulus (cells wholly inside the
// inner radius are skipped), 32 candidates at a time, one per lane, and calls f(in, k, dx, dy) on
// every lane of the warp at every step (warp-uniform), with in = whether galaxy k's squared
// separation r2 lies in [r2lo, r2hi). Must be called by the whole warp.
template <typename F>
__device__ __forceinline__ void for_each_in_annulus(const GridDesc& g, const int32_t* __restrict__ cell_start,
                                                    const int2* __restrict__ pos, long long px, long long py,
                                                    long long r2lo, long long r2hi, int z, int lane, F&& f)
{
    const long long R = isqrt_floor(r2hi - 1);
    const long long ya = max(0LL, fdiv(py - R - g.y0, g.side));
    const long long yb = min((long long)g.ncy - 1, fdiv(py + R - g.y0, g.side));
    for (long long yy = ya; yy <= yb; ++yy) {
        const long long ylo = g.y0 + yy * g.side, yhi = ylo + g.side - 1;
        const long long dymin = max(0LL, max(ylo - py, py - yhi));
        const long long dymax = max(llabs(ylo - py), llabs(yhi - py));
        if (dymin * dymin > r2hi - 1) continue;
        const long long dxo = isqrt_floor(r2hi - 1 - dymin * dymin);
        long long ca = fdiv(px - dxo - g.x0, g.side), cb = fdiv(px + dxo - g.x0, g.side);
        if (cb < 0 || ca > g.ncx - 1) continue;
        ca = max(ca, 0LL);
        cb = min(cb, (long long)g.ncx - 1);
        long long cl = cb + 1, cr = cb;
        if (r2lo - 1 - dymax * dymax >= 0) {
            const long long hx = isqrt_floor(r2lo - 1 - dymax * dymax);
            cl = -fdiv(-(px - hx - g.x0), g.side);      // first cell starting at >= px - hx
            cr = fdiv(px + hx - g.x0 + 1, g.side) - 1;  // last cell ending at <= px + hx
        }
        long long segs[2][2];
        int nseg = 0;
        if (cl <= cr && cl <= cb && cr >= ca) {
            if (ca <= cl - 1) { segs[nseg][0] = ca; segs[nseg][1] = cl - 1; ++nseg; }
            if (cr + 1 <= cb) { segs[nseg][0] = cr + 1; segs[nseg][1] = cb; ++nseg; }
        } else {
            segs[0][0] = ca;
            segs[0][1] = cb;
            nseg = 1;
        }
        const size_t key0 = (size_t)z * g.ncells + (size_t)yy * g.ncx;
        for (int sgi = 0; sgi < nseg; ++sgi) {
            const int k0 = cell_start[key0 + segs[sgi][0]];
            const int k1 = cell_start[key0 + segs[sgi][1] + 1];
            for (int kb = k0; kb < k1; kb += 32) {
                const int k = kb + lane;
                long long dx = 0, dy = 0;
                bool in = false;
                if (k < k1) {
                    const int2 qk = pos[k];
                    dx = (long long)qk.x - px;
                    dy = (long long)qk.y - py;
                    const long long r2 = dx * dx + dy * dy;
                    in = r2 >= r2lo && r2 < r2hi;
                }
                f(in, k, dx, dy);
            }
        }
    }
}

// warp per centre (grid-stride); per bin the warp stages the centre's adjoint moments of every Z
// in shared memory and walks the annulus. The members found are queued (unit vector, galaxy) in
// the warp's shared-memory queue and evaluated 32 at a time, one per lane, so that no lane idles
// through the polynomial evaluations while others hold a member.
constexpr int kQueue = 64;

template <typename T>
__global__ void __launch_bounds__(kPairWarps * 32) moments_adjoint_pairs(const AdjArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = a.nb, nz = a.nz, nmax = a.n_max, nbp = nb_pad(nb);
    const int MG = 2 * nmax + 3, MW = 2 * nmax + 1, o = nmax + 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    cx<T>* co = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)warp * nz * (MG + MW);  // [z][MG + MW]
    cx<T>* qz = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)kPairWarps * nz * (MG + MW) + (size_t)warp * kQueue;
    int* qk = reinterpret_cast<int*>(reinterpret_cast<cx<T>*>(smem_raw) + (size_t)kPairWarps * nz * (MG + MW) +
                                     (size_t)kPairWarps * kQueue) + warp * kQueue;
    const size_t plane = (size_t)a.n_centres * nz * nbp;
    for (int c = blockIdx.x * kPairWarps + warp; c < a.n_centres; c += gridDim.x * kPairWarps) {
        const int d = a.centre_idx[c];
        const int2 p = a.pos[d];
        for (int b = 0; b < nb; ++b) {
            __syncwarp();
            for (int i = lane; i < nz * (MG + MW); i += 32) {
                const int z = i / (MG + MW), qq = i % (MG + MW);
                co[i] = qq < MG ? a.gG[(size_t)qq * plane + ((size_t)c * nz + z) * nbp + b]
                                : a.gW[(size_t)(qq - MG) * plane + ((size_t)c * nz + z) * nbp + b];
            }
            __syncwarp();
            for (int z = 0; z < nz; ++z) {
                const cx<T>* gg = co + (size_t)z * (MG + MW);
                const cx<T>* gw = gg + MG;
                // grad v_k += sum_m gG_m e^{-i m phi}, grad w_k += Re sum_m gW_m e^{-i m phi} for the
                // queued member e
                auto eval = [&](int e) {
                    const cx<T> zz = qz[e];
                    const int k = qk[e];
                    const cx<T> u{zz.x, -zz.y};
                    // m >= 0 part of sum_m gG_m u^m (Horner in u, P <- P u + c: four FMAs)
                    cx<T> P{T(0), T(0)};
#pragma unroll 4
                    for (int mm = nmax - 1; mm >= 0; --mm) P = horner_step(P, u, gg[o + mm]);
                    // m < 0 part: sum_{j >= 1} gG_{-j} z^j = z (gG_{-1} + z (gG_{-2} + ...))
                    cx<T> Q = gg[o - (nmax + 3)];
#pragma unroll 4
                    for (int j = nmax + 2; j >= 1; --j) Q = horner_step(Q, zz, gg[o - j]);
                    Q = cmul(Q, zz);
                    // W: sum_m gW_m u^m
                    cx<T> Rw{T(0), T(0)};
#pragma unroll 4
                    for (int mm = 2 * nmax; mm >= 0; --mm) Rw = horner_step(Rw, u, gw[mm]);
                    atomic_add_vw(a.gvw + 4 * (size_t)k, P.x + Q.x, P.y + Q.y, Rw.x);
                };
                int qn = 0;  // queued members (warp-uniform), < 32 between steps
                for_each_in_annulus(a.g, a.cell_start, a.pos, p.x, p.y, a.e2q[b], a.e2q[b + 1], z, lane,
                                    [&](bool in, int k, long long dx, long long dy) {
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int slot = qn + __popc(m & lt_mask);
                        qz[slot] = unit_dir<T>(dx, dy);
                        qk[slot] = k;
                    }
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        eval(lane);
                        __syncwarp();
                        if (lane < qn - 32) {
                            qz[lane] = qz[32 + lane];
                            qk[lane] = qk[32 + lane];
                        }
                        __syncwarp();
                        qn -= 32;
                    }
                });
                __syncwarp();
                if (lane < qn) eval(lane);
                __syncwarp();
            }
        }
    }
}

// caller order, v = w (gamma_1 + i gamma_2): dL/dgamma_1 = w Re grad v, dL/dgamma_2 = w Im grad v,
// dL/dw = (direct) + Re grad v gamma_1 + Im grad v gamma_2; ADDS to the caller's arrays
template <typename T>
__global__ void adjoint_finish(int64_t n, const int* __restrict__ perm, const T* __restrict__ gvw,
                               const float* __restrict__ g1, const float* __restrict__ g2,
                               const float* __restrict__ w, float* __restrict__ dg1, float* __restrict__ dg2,
                               float* __restrict__ dw)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[d];
        const T vr = gvw[4 * d], vi = gvw[4 * d + 1];
        const T wi = (T)w[i];
        if (dg1) dg1[i] += (float)(wi * vr);
        if (dg2) dg2[i] += (float)(wi * vi);
        if (dw) dw[i] += (float)(gvw[4 * d + 2] + vr * (T)g1[i] + vi * (T)g2[i]);
    }
}

// ------------------------------------------------------------------ exclude_degenerate

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per (centre, z, bin) the sums over neighbours k of redshift bin z in the bin that the j = k
// triplets contribute (u = e^{-i phi}, v = w gamma): D6 = sum v^2 u^6, D2 = sum v^2 u^2,
// E2 = sum |v|^2 u^2, F = sum w^2, written as 4 complex values (F in the real part).
template <typename T>
__global__ void __launch_bounds__(kPairWarps * 32) degenerate_moments(const AdjArgs<T> a, cx<T>* __restrict__ out)
{
    const int nb = a.nb, nz = a.nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = blockIdx.x * kPairWarps + warp; c < a.n_centres; c += gridDim.x * kPairWarps) {
        const int2 p = a.pos[a.centre_idx[c]];
        for (int b = 0; b < nb; ++b)
            for (int z = 0; z < nz; ++z) {
                T s[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
                for_each_in_annulus(a.g, a.cell_start, a.pos, p.x, p.y, a.e2q[b], a.e2q[b + 1], z, lane,
                                    [&](bool in, int k, long long dx, long long dy) {
                    if (!in) return;
                    const cx<T> zz = unit_dir<T>(dx, dy);
                    const cx<T> u{zz.x, -zz.y};
                    const cx<T> u2 = cmul(u, u), u6 = cmul(cmul(u2, u2), u2);
                    const Pay<T> pk = a.pay[k];
                    const cx<T> v{pk.a, pk.b};
                    const cx<T> v2 = cmul(v, v);
                    const T vv = pk.a * pk.a + pk.b * pk.b;
                    const cx<T> d6 = cmul(v2, u6), d2 = cmul(v2, u2);
                    s[0] += d6.x;
                    s[1] += d6.y;
                    s[2] += d2.x;
                    s[3] += d2.y;
                    s[4] += vv * u2.x;
                    s[5] += vv * u2.y;
                    s[6] += pk.w * pk.w;
                });
                for (int i = 0; i < 7; ++i) s[i] = warp_sum(s[i]);
                if (lane == 0) {
                    cx<T>* o = out + (((size_t)c * nz + z) * nb + b) * 4;
                    o[0] = cx<T>{s[0], s[1]};
                    o[1] = cx<T>{s[2], s[3]};
                    o[2] = cx<T>{s[4], s[5]};
                    o[3] = cx<T>{s[6], T(0)};
                }
            }
    }
}

// Block per (z1, z, bin): S0 = sum_i v_i D6, S1 = sum_i conj(v_i) D2, S2 = sum_i v_i E2,
// SN = sum_i w_i F over the centres of redshift bin z1 (FP64, fixed order), then for the triplet
// (z1, z, z) and b1 = b2 = bin, every order: Upsilon_0 += S0, Upsilon_1 += S1, Upsilon_2,3 += S2,
// N -= SN (the j = k terms of the paper's sums, removed).
template <typename T>
__global__ void __launch_bounds__(256) degenerate_correct(const AdjArgs<T> a, const cx<T>* __restrict__ dm,
                                                         double* __restrict__ ups, double* __restrict__ norm)
{
    const int nb = a.nb, nz = a.nz, nmax = a.n_max, NN = nmax + 1, NW = 2 * nmax + 1;
    const int b = blockIdx.x % nb, z = (blockIdx.x / nb) % nz, z1 = blockIdx.x / (nb * nz);
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int c = threadIdx.x; c < a.n_centres; c += blockDim.x) {
        const int d = a.centre_idx[c];
        if ((a.zs ? (int)a.zs[d] : 0) != z1) continue;
        const Pay<T> pv = a.pay[d];
        const cx<double> v{(double)pv.a, (double)pv.b};
        const cx<T>* m = dm + (((size_t)c * nz + z) * nb + b) * 4;
        const cx<double> d6{(double)m[0].x, (double)m[0].y}, d2{(double)m[1].x, (double)m[1].y};
        const cx<double> e2{(double)m[2].x, (double)m[2].y};
        const cx<double> t0 = cmul(v, d6), t1 = cmul(cconj(v), d2), t2 = cmul(v, e2);
        s[0] += t0.x; s[1] += t0.y; s[2] += t1.x; s[3] += t1.y; s[4] += t2.x; s[5] += t2.y;
        s[6] += (double)pv.w * (double)m[3].x;
    }
    __shared__ double red[7][256];
    for (int i = 0; i < 7; ++i) red[i][threadIdx.x] = s[i];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int i = 0; i < 7; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + h];
        __syncthreads();
    }
    const int zt = (z1 * nz + z) * nz + z;
    const size_t bb = (size_t)b * nb + b, nbb = (size_t)nb * nb;
    cx<double>* U = reinterpret_cast<cx<double>*>(ups);
    cx<double>* N = reinterpret_cast<cx<double>*>(norm);
    for (int n = threadIdx.x; n < NN; n += blockDim.x) {
        const cx<double> S0{red[0][0], red[1][0]}, S1{red[2][0], red[3][0]}, S2{red[4][0], red[5][0]};
        U[(((size_t)zt * 4 + 0) * NN + n) * nbb + bb] = cadd(U[(((size_t)zt * 4 + 0) * NN + n) * nbb + bb], S0);
        U[(((size_t)zt * 4 + 1) * NN + n) * nbb + bb] = cadd(U[(((size_t)zt * 4 + 1) * NN + n) * nbb + bb], S1);
        U[(((size_t)zt * 4 + 2) * NN + n) * nbb + bb] = cadd(U[(((size_t)zt * 4 + 2) * NN + n) * nbb + bb], S2);
        U[(((size_t)zt * 4 + 3) * NN + n) * nbb + bb] = cadd(U[(((size_t)zt * 4 + 3) * NN + n) * nbb + bb], S2);
    }
    for (int m = threadIdx.x; m < NW; m += blockDim.x) {
        cx<double>& e = N[((size_t)zt * NW + m) * nbb + bb];
        e.x -= red[6][0];
    }
}

// ---- adjoint of the exclude_degenerate correction. The forward adds S0 = sum_i v_i D6_i to every
// order of Upsilon_0, S1 = sum_i v_i^* D2_i to Upsilon_1, S2 = sum_i v_i E2_i to Upsilon_2 and
// Upsilon_3 and subtracts SN = sum_i w_i F_i from Re N (b1 = b2, Z2 = Z3). Block-free pass first:
// per (Z1, z, bin) gS0 = sum_n dL/dUpsilon_0,n, gS1, gS2 (Upsilon_2 and _3) and gSN = -sum_m
// Re dL/dN_m, stored as dgs[(z1 nz + z) nb + b][0..3] (gSN in the real part).
__global__ void degenerate_grad_sums(int nz, int nb, int n_max, const double* __restrict__ gups,
                                     const double* __restrict__ gnorm, cx<double>* __restrict__ dgs)
{
    const int NN = n_max + 1, NW = 2 * n_max + 1;
    const int total = nz * nz * nb;
    const size_t nbb = (size_t)nb * nb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int b = t % nb, z = (t / nb) % nz, z1 = t / (nb * nz);
        const int zt = (z1 * nz + z) * nz + z;
        const size_t bb = (size_t)b * nb + b;
        cx<double> g[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int n = 0; n < NN; ++n)
            for (int mu = 0; mu < 4; ++mu) {
                const size_t i = 2 * ((((size_t)zt * 4 + mu) * NN + n) * nbb + bb);
                const int slot = mu < 3 ? mu : 2;
                g[slot].x += gups[i];
                g[slot].y += gups[i + 1];
            }
        double gn = 0.0;
        for (int m = 0; m < NW; ++m) gn -= gnorm[2 * (((size_t)zt * NW + m) * nbb + bb)];
        dgs[(size_t)t * 4 + 0] = g[0];
        dgs[(size_t)t * 4 + 1] = g[1];
        dgs[(size_t)t * 4 + 2] = g[2];
        dgs[(size_t)t * 4 + 3] = cx<double>{gn, 0.0};
    }
}

// Warp per centre i: per (bin, z) of the neighbours, with u = e^{-i phi_ij},
//   grad v_j += 2 v_j^* (u^6)^* gD6 + 2 v_j^* (u^2)^* gD2 + 2 v_j Re(gE2 (u^2)^*),
//   grad w_j += 2 w_j gF,   gD6 = v_i^* gS0, gD2 = v_i gS1, gE2 = v_i^* gS2, gF = w_i gSN,
// and, with the centre's own sums D6, D2, E2, F (re-formed in the same walk),
//   grad v_i += D6^* gS0 + D2 gS1^* + E2^* gS2,   grad w_i += F gSN.
template <typename T>
__global__ void __launch_bounds__(kPairWarps * 32) degenerate_adjoint_pairs(const AdjArgs<T> a)
{
    const int nb = a.nb, nz = a.nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = blockIdx.x * kPairWarps + warp; c < a.n_centres; c += gridDim.x * kPairWarps) {
        const int d = a.centre_idx[c];
        const int2 p = a.pos[d];
        const int z1 = a.zs ? (int)a.zs[d] : 0;
        const Pay<T> pv = a.pay[d];
        const cx<double> vi{(double)pv.a, (double)pv.b};
        const double wi = (double)pv.w;
        double cgr = 0.0, cgi = 0.0, cgw = 0.0;  // the centre's own gradient (lane 0 adds it)
        for (int b = 0; b < nb; ++b)
            for (int z = 0; z < nz; ++z) {
                const cx<double>* gs = a.dgs + ((size_t)(z1 * nz + z) * nb + b) * 4;
                const cx<double> gS0 = gs[0], gS1 = gs[1], gS2 = gs[2];
                const double gSN = gs[3].x;
                const cx<double> gD6 = cmul(cconj(vi), gS0), gD2 = cmul(vi, gS1), gE2 = cmul(cconj(vi), gS2);
                const double gF = wi * gSN;
                double sd[7] = {0, 0, 0, 0, 0, 0, 0};  // this lane's share of D6, D2, E2, F
                for_each_in_annulus(a.g, a.cell_start, a.pos, p.x, p.y, a.e2q[b], a.e2q[b + 1], z, lane,
                                    [&](bool in, int k, long long dx, long long dy) {
                    if (!in) return;
                    const cx<T> zz = unit_dir<T>(dx, dy);
                    const cx<double> u{(double)zz.x, -(double)zz.y};
                    const cx<double> u2 = cmul(u, u), u6 = cmul(cmul(u2, u2), u2);
                    const Pay<T> pk = a.pay[k];
                    const cx<double> vj{(double)pk.a, (double)pk.b};
                    const double wj = (double)pk.w;
                    const cx<double> vj2 = cmul(vj, vj);
                    const cx<double> d6 = cmul(vj2, u6), d2 = cmul(vj2, u2);
                    const double vv = vj.x * vj.x + vj.y * vj.y;
                    sd[0] += d6.x;
                    sd[1] += d6.y;
                    sd[2] += d2.x;
                    sd[3] += d2.y;
                    sd[4] += vv * u2.x;
                    sd[5] += vv * u2.y;
                    sd[6] += wj * wj;
                    const cx<double> t6 = cmul(cmul(cconj(vj), cconj(u6)), gD6);
                    const cx<double> t2 = cmul(cmul(cconj(vj), cconj(u2)), gD2);
                    const double re = cmul(gE2, cconj(u2)).x;
                    atomic_add_vw(a.gvw + 4 * (size_t)k, (T)(2.0 * (t6.x + t2.x + vj.x * re)),
                                  (T)(2.0 * (t6.y + t2.y + vj.y * re)), (T)(2.0 * wj * gF));
                });
                for (int i = 0; i < 7; ++i) sd[i] = warp_sum(sd[i]);
                const cx<double> D6{sd[0], sd[1]}, D2{sd[2], sd[3]}, E2{sd[4], sd[5]};
                const cx<double> gv = cadd(cadd(cmul(cconj(D6), gS0), cmul(D2, cconj(gS1))), cmul(cconj(E2), gS2));
                cgr += gv.x;
                cgi += gv.y;
                cgw += sd[6] * gSN;
            }
        if (lane == 0) atomic_add_vw(a.gvw + 4 * (size_t)d, (T)cgr, (T)cgi, (T)cgw);
    }
}

template <typename T>
static cudaError_t run_degenerate(const AdjArgs<T>& a, cx<T>* scratch, double* ups, double* norm, int n_sm,
                                  cudaStream_t st)
{
    if (a.n_centres <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((a.n_centres + kPairWarps - 1) / kPairWarps, (int64_t)n_sm * 32);
    degenerate_moments<T><<<blocks, kPairWarps * 32, 0, st>>>(a, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    degenerate_correct<T><<<a.nz * a.nz * a.nb, 256, 0, st>>>(a, scratch, ups, norm);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run(const AdjArgs<T>& a, int64_t n, const int* perm, const float* g1, const float* g2,
                       const float* w, float* dg1, float* dg2, float* dw, int n_sm, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.gvw, 0, sizeof(T) * 4 * (size_t)n, st);
    if (e != cudaSuccess) return e;
    if (a.n_centres > 0) {
        const int MG = 2 * a.n_max + 3, MW = 2 * a.n_max + 1;
        dim3 g1d((a.n_centres + kTileC - 1) / kTileC, MG + MW);
        const int64_t z3 = (int64_t)a.nz * a.nz * a.nz, nbb = (int64_t)a.nb * a.nb;
        const int64_t nU = z3 * 4 * (a.n_max + 1), tot = (nU + z3 * (2 * a.n_max + 1)) * nbb;
        grad_tables<T><<<(unsigned)std::min<int64_t>((tot + 255) / 256, (int64_t)n_sm * 16), 256, 0, st>>>(a, nU, tot);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        contract_adjoint_moments<T><<<g1d, 256, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const size_t sm_coef = sizeof(cx<T>) * (size_t)a.nb * a.nb;
        e = set_smem_attr(contract_adjoint_coef<T>, sm_coef);
        if (e != cudaSuccess) return e;
        constexpr int per_block = kCoefWarps * kCoefCentres;
        contract_adjoint_coef<T><<<(a.n_centres + per_block - 1) / per_block, kCoefWarps * 32, sm_coef, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const size_t sm_pair = sizeof(cx<T>) * (size_t)kPairWarps * (a.nz * (MG + MW) + kQueue) +
                               sizeof(int) * (size_t)kPairWarps * kQueue;
        e = set_smem_attr(moments_adjoint_pairs<T>, sm_pair);
        if (e != cudaSuccess) return e;
        const int blocks = (int)std::min<int64_t>((a.n_centres + kPairWarps - 1) / kPairWarps, (int64_t)n_sm * 32);
        moments_adjoint_pairs<T><<<blocks, kPairWarps * 32, sm_pair, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.dgs && a.n_centres > 0) {
        // the j = k triplets left out of the forward (exclude_degenerate)
        const int total = a.nz * a.nz * a.nb;
        degenerate_grad_sums<<<(total + 127) / 128, 128, 0, st>>>(a.nz, a.nb, a.n_max, a.gups, a.gnorm, a.dgs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int blocks = (int)std::min<int64_t>((a.n_centres + kPairWarps - 1) / kPairWarps, (int64_t)n_sm * 32);
        degenerate_adjoint_pairs<T><<<blocks, kPairWarps * 32, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 16));
    adjoint_finish<T><<<gb, 256, 0, st>>>(n, perm, a.gvw, g1, g2, w, dg1, dg2, dw);
    return cudaGetLastError();
}

}  // namespace adj

cudaError_t launch_moments_adjoint_f32(const AdjArgs<float>& a, int64_t n, const int* perm, const float* g1,
                                       const float* g2, const float* w, float* dg1, float* dg2, float* dw,
                                       int n_sm, cudaStream_t st)
{
    return adj::run<float>(a, n, perm, g1, g2, w, dg1, dg2, dw, n_sm, st);
}

cudaError_t launch_moments_adjoint_f64(const AdjArgs<double>& a, int64_t n, const int* perm, const float* g1,
                                       const float* g2, const float* w, float* dg1, float* dg2, float* dw,
                                       int n_sm, cudaStream_t st)
{
    return adj::run<double>(a, n, perm, g1, g2, w, dg1, dg2, dw, n_sm, st);
}

}  // namespace mp3

namespace mp3 {

cudaError_t launch_degenerate_f32(const AdjArgs<float>& a, void* scratch, double* ups, double* norm, int n_sm,
                                  cudaStream_t st)
{
    return adj::run_degenerate<float>(a, reinterpret_cast<cx<float>*>(scratch), ups, norm, n_sm, st);
}

cudaError_t launch_degenerate_f64(const AdjArgs<double>& a, void* scratch, double* ups, double* norm, int n_sm,
                                  cudaStream_t st)
{
    return adj::run_degenerate<double>(a, reinterpret_cast<cx<double>*>(scratch), ups, norm, n_sm, st);
}

}  // namespace mp3
