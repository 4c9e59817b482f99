// Grid moments of the combined estimator by FFT convolution (paper Sec. 3.2: on a regular grid the
// moments G_n^Delta and W_n^Delta of every pixel are convolutions of the gridded fields w gamma and
// w with the bin kernels e^{i n phi} 1[theta in bin], which the paper evaluates with FFTs).
//
// The fields are those of the pixel catalog of the direct form (csrc/grid.cu): each pixel with
// weight W > 0 carries v = W (sum w gamma / W) and W, rounded to float32 and multiplied in the
// moment precision exactly as the pixel catalog's payload is, at the pixel centre. The kernel of
// bin b and order m at a pixel offset d = (dx, dy) is 1[e_b^2 <= |d|^2 pq^2 < e_{b+1}^2] z^m with
// z = (dx + i dy) / |d|, the exact integer bin test of the pixel-pair sums, so for the pixels that
// hold centres the result equals those sums up to the FFT's rounding. With the fields zero-padded
// by the largest offset of the level's bins the circular convolution is the linear one:
//   G_m(p, z, b) = sum_q F_z(q) K_{b,m}(q - p) = (F_z (*) K'_{b,m})(p),  K'(u) = K(-u).
// Per batch of orders m >= 0 the kernels of every bin of the level are built on the padded grid
// and transformed (one batched cuFFT plan); since K_{-m} = conj(K_m), the spectrum of the order -m
// kernel is conj(K^_m(-k)), so one transform serves G_m, G_{-m} and W_m. Each use multiplies by a
// neighbour z-bin's field spectrum, transforms back, and writes the values at the centres' pixels
// into the centres' moment rows, all bins of the level at once (whole runs of bins per row). cuFFT
// plans are cached per (grid, batch, precision) in a cache owned by the context.
#include <cufft.h>

#include <map>
#include <tuple>

#include "common.cuh"

namespace mp3 {

struct FftPlanCache {
    std::map<std::tuple<int, int, int, int>, cufftHandle> plans;
    ~FftPlanCache()
    {
        for (auto& kv : plans) cufftDestroy(kv.second);
    }
};

FftPlanCache* fft_cache_create() { return new FftPlanCache(); }
void fft_cache_destroy(FftPlanCache* c) { delete c; }

#ifndef MP3_FFT_MAX35
#define MP3_FFT_MAX35 99  // largest power of 3 and of 5 allowed in a transform length
#endif

// smallest length >= n of the form 2^a 3^b 5^c (b, c <= MP3_FFT_MAX35): fast cuFFT sizes
static int fft_len(int n)
{
    for (int m = n;; ++m) {
        int r = m, e3 = 0, e5 = 0;
        while (r % 2 == 0) r /= 2;
        while (r % 3 == 0) r /= 3, ++e3;
        while (r % 5 == 0) r /= 5, ++e5;
        if (r == 1 && e3 <= MP3_FFT_MAX35 && e5 <= MP3_FFT_MAX35) return m;
    }
}

template <typename T>
struct FftType;
template <>
struct FftType<float> {
    using C = cufftComplex;
    static constexpr cufftType kType = CUFFT_C2C;
    static cufftResult exec(cufftHandle h, void* data, int dir)
    {
        return cufftExecC2C(h, (C*)data, (C*)data, dir);
    }
};
template <>
struct FftType<double> {
    using C = cufftDoubleComplex;
    static constexpr cufftType kType = CUFFT_Z2Z;
    static cufftResult exec(cufftHandle h, void* data, int dir)
    {
        return cufftExecZ2Z(h, (C*)data, (C*)data, dir);
    }
};

template <typename T>
static cufftHandle get_plan(FftPlanCache* cache, int ny, int nx, int batch, cudaStream_t st, cufftResult* err)
{
    const auto key = std::make_tuple(ny, nx, batch, (int)sizeof(T));
    auto it = cache->plans.find(key);
    cufftHandle h = 0;
    if (it != cache->plans.end()) {
        h = it->second;
    } else {
        int dims[2] = {ny, nx};
        *err = cufftPlanMany(&h, 2, dims, nullptr, 1, ny * nx, nullptr, 1, ny * nx, FftType<T>::kType, batch);
        if (*err != CUFFT_SUCCESS) return 0;
        cache->plans[key] = h;
    }
    *err = cufftSetStream(h, st);
    return h;
}

// fields [2][nz][NY][NX]: v (w gamma) then w, the pixel catalog's payload on the padded grid
template <typename T>
__global__ void k_fft_fields(int nz, int npx, int npy, int NX, int NY, const double* __restrict__ s,
                             cx<T>* __restrict__ f)
{
    const int64_t plane = (int64_t)NX * NY, total = (int64_t)nz * plane;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(t / plane);
        const int64_t r = t - (int64_t)z * plane;
        const int iy = (int)(r / NX), ix = (int)(r - (int64_t)iy * NX);
        cx<T> v{T(0), T(0)}, w{T(0), T(0)};
        if (ix < npx && iy < npy) {
            const int64_t p = ((int64_t)z * npy + iy) * npx + ix;
            const double W = s[3 * p];
            if (W > 0.0) {
                const float pw = (float)W, pg1 = (float)(s[3 * p + 1] / W), pg2 = (float)(s[3 * p + 2] / W);
                v = cx<T>{(T)pw * (T)pg1, (T)pw * (T)pg2};
                w = cx<T>{(T)pw, T(0)};
            }
        }
        f[t] = v;
        f[total + t] = w;
    }
}

// kernels K'_{b,m}(u) = K_{b,m}(-u) of the bins b0 .. b0 + nbr - 1 and orders m = m0 .. m0 + nk - 1
// on the padded grid [nbr][nk][NY][NX]; u wraps around the grid (offsets up to R pixels each way)
template <typename T>
__global__ void k_fft_kernels(int NX, int NY, int R, long long pq, const long long* __restrict__ e2q, int nbr, int m0,
                              int nk, cx<T>* __restrict__ K)
{
    const int64_t plane = (int64_t)NX * NY, total = (int64_t)nbr * nk * plane;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int bj = (int)(t / plane);
        const int bb = bj / nk, j = bj - bb * nk;
        const int64_t r = t - (int64_t)bj * plane;
        const int iy = (int)(r / NX), ix = (int)(r - (int64_t)iy * NX);
        const int ux = ix <= NX / 2 ? ix : ix - NX, uy = iy <= NY / 2 ? iy : iy - NY;
        cx<T> k{T(0), T(0)};
        if (ux >= -R && ux <= R && uy >= -R && uy <= R) {
            const long long dx = -ux, dy = -uy;  // the kernel at -u
            const long long r2 = (dx * dx + dy * dy) * pq * pq;
            if (r2 >= e2q[bb] && r2 < e2q[bb + 1]) {
                double sn, cs;
                sincos((double)(m0 + j) * atan2((double)dy, (double)dx), &sn, &cs);
                k = cx<T>{(T)cs, (T)sn};
            }
        }
        K[t] = k;
    }
}

// P[i] = F * K^[i] for the nbr * nk spectra, or with flip F * conj(K^[i](-k)) (the order -m kernel)
template <typename T>
__global__ void k_fft_mul(int NX, int NY, int n, bool flip, const cx<T>* __restrict__ F, const cx<T>* __restrict__ K,
                          cx<T>* __restrict__ P)
{
    const int64_t plane = (int64_t)NX * NY, total = (int64_t)n * plane;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / plane, r = t - i * plane;
        cx<T> k;
        if (flip) {
            const int iy = (int)(r / NX), ix = (int)(r - (int64_t)iy * NX);
            const int fy = iy == 0 ? 0 : NY - iy, fx = ix == 0 ? 0 : NX - ix;
            k = cconj(K[i * plane + (int64_t)fy * NX + fx]);
        } else {
            k = K[t];
        }
        P[t] = cmul(F[r], k);
    }
}

// each centre's pixel on the padded grid (iy NX + ix), or -1 when that pixel has no weight (it is
// not in the pixel catalog of the direct form, whose grid bins are then zero)
__global__ void k_fft_centre_pixels(int64_t nc, const int* __restrict__ centre_idx, const int2* __restrict__ pos,
                                    const uint8_t* __restrict__ zs, long long x0, long long y0, long long pq, int npx,
                                    int npy, int NX, const double* __restrict__ s, int* __restrict__ cpx)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = centre_idx[c];
        const int2 p = pos[i];
        const long long dx = (long long)p.x - x0, dy = (long long)p.y - y0;
        const int ix = (int)min(max(dx < 0 ? -1LL : dx / pq, 0LL), (long long)npx - 1);
        const int iy = (int)min(max(dy < 0 ? -1LL : dy / pq, 0LL), (long long)npy - 1);
        const int zc = zs ? (int)zs[i] : 0;
        const bool has = s[3 * (((int64_t)zc * npy + iy) * npx + ix)] > 0.0;
        cpx[c] = has ? iy * NX + ix : -1;
    }
}

// moment rows of every centre: for the orders j0 .. j1 - 1 of a batch of nk, order slot
// slot0 + dir j, neighbour z-bin z, bins b0 .. b0 + nbr - 1 (P [nbr][nk][NY][NX]): the convolution
// at the centre's pixel (normalised), zero for the centres without one. One thread per (order,
// centre) writes its run of bins.
template <typename T>
__global__ void k_fft_gather(int64_t nc, int nk, int j0, int j1, int nbr, const int* __restrict__ cpx, int64_t grid_plane,
                             const cx<T>* __restrict__ P, T scale, int slot0, int dir, size_t plane_rows, int nz,
                             int z, int nbp, int b0, cx<T>* __restrict__ out)
{
    // one output element per thread, the level's bins of a centre on consecutive threads, so a
    // warp writes whole runs of each centre's row
    const int64_t total = (int64_t)(j1 - j0) * nc * nbr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / nbr;
        const int bb = (int)(t - q * nbr);
        const int j = j0 + (int)(q / nc);
        const int64_t c = q - (int64_t)(j - j0) * nc;
        const int px = cpx[c];
        cx<T> v{T(0), T(0)};
        if (px >= 0) {
            const cx<T> g = P[((int64_t)bb * nk + j) * grid_plane + px];
            v = cx<T>{g.x * scale, g.y * scale};
        }
        out[(size_t)(slot0 + dir * j) * plane_rows + ((size_t)c * nz + z) * nbp + b0 + bb] = v;
    }
}

static unsigned fft_blocks(int64_t m, int n_sm)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)n_sm * 16));
}

template <typename T>
cudaError_t grid_fft_moments(FftPlanCache* cache, int64_t nc, int nz, int nb, int b0, int b1, int n_max,
                             const long long* h_e2q, const int* centre_idx, const int2* pos, const uint8_t* zs,
                             long long x0, long long y0, long long pq, int npx, int npy, const double* gridsum,
                             void* work, size_t work_bytes, cx<T>* G, cx<T>* W, int n_sm, cudaStream_t st,
                             const char** what)
{
    if (nc <= 0 || b1 <= b0) return cudaSuccess;
    const int nbr = b1 - b0;
    // the largest pixel offset of the level's bins, and the padded grid
    const double rmax = std::sqrt((double)h_e2q[b1]) / (double)pq;
    const int R = (int)std::ceil(rmax) + 1;
    const int NX = fft_len(npx + R + 1), NY = fft_len(npy + R + 1);
    const int64_t plane = (int64_t)NX * NY;
    const size_t pbytes = sizeof(cx<T>) * (size_t)plane;
    const int nbp = nb_pad(nb);
    const size_t plane_rows = (size_t)nc * nz * nbp;
    // work: the level's squared edges, the centres' pixels, fields [2 nz], kernel spectra
    // [nbr][nk], products [nbr][nk]
    const size_t head = 1024 + ((sizeof(int) * (size_t)nc + 255) / 256) * 256;
    const size_t field_bytes = 2 * (size_t)nz * pbytes;
    if (work_bytes < head + field_bytes + 2 * (size_t)nbr * pbytes) {
        *what = "FFT workspace too small";
        return cudaErrorMemoryAllocation;
    }
    const int mtop = 2 * n_max > n_max + 3 ? 2 * n_max : n_max + 3;  // orders |m| <= mtop are needed
    const int nk_max = (int)std::min<size_t>((size_t)mtop + 1, (work_bytes - head - field_bytes) / (2 * (size_t)nbr * pbytes));
    long long* e2q = reinterpret_cast<long long*>(work);
    int* cpx = reinterpret_cast<int*>(static_cast<char*>(work) + 1024);
    cx<T>* F = reinterpret_cast<cx<T>*>(static_cast<char*>(work) + head);
    cx<T>* K = F + 2 * (int64_t)nz * plane;
    cx<T>* P = K + (int64_t)nbr * nk_max * plane;
    cufftResult fr = CUFFT_SUCCESS;
    cudaError_t e = cudaMemcpyAsync(e2q, h_e2q + b0, sizeof(long long) * (nbr + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;

    k_fft_fields<T><<<fft_blocks((int64_t)nz * plane, n_sm), 256, 0, st>>>(nz, npx, npy, NX, NY, gridsum, F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_fft_centre_pixels<<<fft_blocks(nc, n_sm), 256, 0, st>>>(nc, centre_idx, pos, zs, x0, y0, pq, npx, npy, NX,
                                                              gridsum, cpx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cufftHandle hf = get_plan<T>(cache, NY, NX, 2 * nz, st, &fr);
    if (fr != CUFFT_SUCCESS || FftType<T>::exec(hf, F, CUFFT_FORWARD) != CUFFT_SUCCESS) {
        *what = "cuFFT of the fields failed";
        return cudaErrorUnknown;
    }
    const T scale = (T)(1.0 / (double)plane);
    // G slot of order m: m + n_max + 3 (m = -n_max-3 .. n_max-1); W slot: m (m = 0 .. 2 n_max)
    for (int m0 = 0; m0 <= mtop; m0 += nk_max) {
        const int nk = std::min(nk_max, mtop - m0 + 1);
        k_fft_kernels<T><<<fft_blocks((int64_t)nbr * nk * plane, n_sm), 256, 0, st>>>(NX, NY, R, pq, e2q, nbr, m0, nk,
                                                                                      K);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cufftHandle hk = get_plan<T>(cache, NY, NX, nbr * nk, st, &fr);
        if (fr != CUFFT_SUCCESS || FftType<T>::exec(hk, K, CUFFT_FORWARD) != CUFFT_SUCCESS) {
            *what = "cuFFT of the bin kernels failed";
            return cudaErrorUnknown;
        }
        // uses of the batch: G_{+m} (m <= n_max - 1), G_{-m} (1 <= m <= n_max + 3), W_m (m <= 2 n_max)
        for (int use = 0; use < 3; ++use) {
            int mlo = m0, mhi = m0 + nk - 1;
            if (use == 0) mhi = std::min(mhi, n_max - 1);
            if (use == 1) mlo = std::max(mlo, 1), mhi = std::min(mhi, n_max + 3);
            if (use == 2) mhi = std::min(mhi, 2 * n_max);
            if (mlo > mhi) continue;
            const int j0 = mlo - m0, jn = mhi - m0 + 1;  // orders of the batch this use writes
            const int slot0 = use == 0 ? m0 + n_max + 3 : use == 1 ? n_max + 3 - m0 : m0;
            const int dir = use == 1 ? -1 : 1;
            cx<T>* out = use == 2 ? W : G;
            for (int z = 0; z < nz; ++z) {
                const cx<T>* Fz = F + ((int64_t)(use == 2 ? nz : 0) + z) * plane;
                k_fft_mul<T><<<fft_blocks((int64_t)nbr * nk * plane, n_sm), 256, 0, st>>>(NX, NY, nbr * nk, use == 1,
                                                                                          Fz, K, P);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                if (FftType<T>::exec(hk, P, CUFFT_INVERSE) != CUFFT_SUCCESS) {
                    *what = "inverse cuFFT failed";
                    return cudaErrorUnknown;
                }
                k_fft_gather<T><<<fft_blocks((int64_t)(jn - j0) * nc * nbr, n_sm), 256, 0, st>>>(
                    nc, nk, j0, jn, nbr, cpx, plane, P, scale, slot0, dir, plane_rows, nz, z, nbp, b0, out);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

// workspace for a level of nbr bins: the fields and the kernel and product arrays of at least one
// order per bin; up to max_orders orders per batch as the budget allows
size_t grid_fft_work_bytes(int64_t nc, int nz, int nbr, int npx, int npy, double rmax_pixels, size_t elem_bytes,
                           int max_orders, size_t budget)
{
    const int R = (int)std::ceil(rmax_pixels) + 1;
    const size_t plane = (size_t)fft_len(npx + R + 1) * fft_len(npy + R + 1);
    const size_t pbytes = 2 * elem_bytes * plane;
    const size_t head = 1024 + ((sizeof(int) * (size_t)nc + 255) / 256) * 256;
    const size_t need = head + (2 * (size_t)nz + 2 * (size_t)nbr) * pbytes;
    const size_t want = head + (2 * (size_t)nz + 2 * (size_t)nbr * max_orders) * pbytes;
    return std::max(need, std::min(want, budget));
}

template cudaError_t grid_fft_moments<float>(FftPlanCache*, int64_t, int, int, int, int, int, const long long*,
                                             const int*, const int2*, const uint8_t*, long long, long long, long long,
                                             int, int, const double*, void*, size_t, cx<float>*, cx<float>*, int,
                                             cudaStream_t, const char**);
template cudaError_t grid_fft_moments<double>(FftPlanCache*, int64_t, int, int, int, int, int, const long long*,
                                              const int*, const int2*, const uint8_t*, long long, long long,
                                              long long, int, int, const double*, void*, size_t, cx<double>*,
                                              cx<double>*, int, cudaStream_t, const char**);

}  // namespace mp3
