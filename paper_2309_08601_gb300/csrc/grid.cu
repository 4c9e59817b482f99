// The grid-based approximation (paper Sec. 3.2): the catalog's weights w and products w gamma
// are summed per pixel of a regular grid, and each pixel becomes a galaxy at its centre with
// weight W = sum w and shear (sum w gamma) / W. The moments of the pixel catalog are the grid
// moments G_n^Delta, W_n^Delta of the paper (its convolutions of the gridded fields with the bin
// kernels e^{i n phi} 1[theta in Theta], here evaluated by the library's direct sums over pixel
// pairs, the same arithmetic as the convolution), and the contraction of the pixel catalog is
// Eq. UpsilonmuGrid, the outer sum running over pixels.
// Only the non-empty pixels are emitted (flags, an exclusive scan, a scatter), in (z, iy, ix) order.
// The per-pixel sums are taken in FP64 with atomics: a product of two float32 numbers is exact in
// FP64 and so are the sums of a pixel's few products, so the result does not depend on the order
// of the additions.
#include "common.cuh"

namespace mp3 {

__global__ void k_grid_zero(int64_t m, double* __restrict__ s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = 0.0;
}

// pixel (ix, iy) of z-bin z covers [origin + i pq, origin + (i + 1) pq) on each axis; positions
// outside the grid are clamped to its edge pixels, z-bins to n_z - 1
__global__ void k_grid_scatter(int64_t n, const int32_t* __restrict__ xq, const int32_t* __restrict__ yq,
                               const float* __restrict__ g1, const float* __restrict__ g2,
                               const float* __restrict__ w, const uint8_t* __restrict__ zb, int nz, long long x0,
                               long long y0, long long pq, int npx, int npy, double* __restrict__ s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const long long dx = (long long)xq[i] - x0, dy = (long long)yq[i] - y0;
        const int ix = (int)min(max(dx < 0 ? -1LL : dx / pq, 0LL), (long long)npx - 1);
        const int iy = (int)min(max(dy < 0 ? -1LL : dy / pq, 0LL), (long long)npy - 1);
        const int z = zb ? min((int)zb[i], nz - 1) : 0;
        const int64_t p = ((int64_t)z * npy + iy) * npx + ix;
        const double wi = (double)w[i];
        atomicAdd(&s[3 * p], wi);
        atomicAdd(&s[3 * p + 1], wi * (double)g1[i]);
        atomicAdd(&s[3 * p + 2], wi * (double)g2[i]);
    }
}

__global__ void k_grid_flags(int64_t npix, const double* __restrict__ s, int* __restrict__ flags)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x)
        flags[p] = s[3 * p] > 0.0 ? 1 : 0;
}

// the non-empty pixels in (z, iy, ix) order, pixel p at rank[p]
__global__ void k_grid_emit(int64_t npix, int npx, int npy, long long x0, long long y0, long long pq,
                            const double* __restrict__ s, const int* __restrict__ rank, int32_t* __restrict__ oxq,
                            int32_t* __restrict__ oyq, float* __restrict__ og1, float* __restrict__ og2,
                            float* __restrict__ ow, uint8_t* __restrict__ ozb)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const double W = s[3 * p];
        if (!(W > 0.0)) continue;
        const int q = rank[p];
        ow[q] = (float)W;
        og1[q] = (float)(s[3 * p + 1] / W);
        og2[q] = (float)(s[3 * p + 2] / W);
        oxq[q] = (int32_t)(x0 + (p % npx) * pq + pq / 2);
        oyq[q] = (int32_t)(y0 + ((p / npx) % npy) * pq + pq / 2);
        if (ozb) ozb[q] = (uint8_t)(p / ((int64_t)npx * npy));
    }
}

// ---- combined estimator (Sec. 3.3): the moments of the bins that use the grid are, for every
// centre galaxy, those of the pixel it lies in (the value G_n^Delta at its pixel, taken as it is:
// Eq. CombinedEstimatorRegridding holds without a division by the galaxies per pixel)

// the pixel of a galaxy at fixed-point (x, y) in z-bin z, by the same rule as k_grid_scatter
__device__ __forceinline__ int64_t grid_pixel(int x, int y, int z, long long x0, long long y0, long long pq,
                                              int npx, int npy)
{
    const long long dx = (long long)x - x0, dy = (long long)y - y0;
    const int ix = (int)min(max(dx < 0 ? -1LL : dx / pq, 0LL), (long long)npx - 1);
    const int iy = (int)min(max(dy < 0 ? -1LL : dy / pq, 0LL), (long long)npy - 1);
    return ((int64_t)z * npy + iy) * npx + ix;
}

// pmask[q] = 1 for the pixels (catalog index q) that hold a centre galaxy; pmask zeroed before
__global__ void k_grid_centre_mask(int64_t nc, const int* __restrict__ centre_idx, const int2* __restrict__ pos,
                                   const uint8_t* __restrict__ zs, long long x0, long long y0, long long pq,
                                   int npx, int npy, const int* __restrict__ flags, const int* __restrict__ rank,
                                   uint8_t* __restrict__ pmask)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int j = centre_idx[c];
        const int2 p = pos[j];
        const int64_t pid = grid_pixel(p.x, p.y, zs ? (int)zs[j] : 0, x0, y0, pq, npx, npy);
        if (flags[pid]) pmask[rank[pid]] = 1;
    }
}

// inv[q] = the moment row of pixel q in the pixel catalog's context (its rows are its centres in
// sorted order; perm maps a sorted position to the catalog index)
__global__ void k_grid_invert(int64_t nrows, const int* __restrict__ centre_idx, const int* __restrict__ perm,
                              int* __restrict__ inv)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x)
        inv[perm[centre_idx[r]]] = (int)r;
}

// srow[c] = the moment row, in the pixel catalog's context, of the pixel centre c lies in, or -1
// when that pixel has no weight (W <= 0, not in the pixel catalog)
__global__ void k_grid_rows(int64_t nc, const int* __restrict__ centre_idx, const int2* __restrict__ pos,
                            const uint8_t* __restrict__ zs, long long x0, long long y0, long long pq, int npx,
                            int npy, const int* __restrict__ flags, const int* __restrict__ rank,
                            const int* __restrict__ inv, int* __restrict__ srow)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int j = centre_idx[c];
        const int2 p = pos[j];
        const int64_t pid = grid_pixel(p.x, p.y, zs ? (int)zs[j] : 0, x0, y0, pq, npx, npy);
        srow[c] = flags[pid] ? inv[rank[pid]] : -1;
    }
}

// rows [b0, b0 + nbr) of G (order slots [0, lg)) and W (slots [0, lw)) of every centre from the
// pixel moments Gs, Ws ([slot][nsub][nz][nbp]), zeros where srow < 0. Order slot q = blockIdx.y;
// the threads run over (centre, z, bin) with the bin fastest, so a warp writes whole runs of
// bins; I is the index type (32-bit when nc nz nbr fits)
template <typename T, typename I>
__global__ void k_grid_copy(I ncz, int nz, int nbp, int b0, int nbr, int lw, const int* __restrict__ srow,
                            int64_t nsub, const cx<T>* __restrict__ Gs, const cx<T>* __restrict__ Ws,
                            cx<T>* __restrict__ G, cx<T>* __restrict__ W)
{
    const int q = blockIdx.y;
    const I total = ncz * (I)nbr;
    const int64_t nc = (int64_t)(ncz / (I)nz);
    for (I t = blockIdx.x * (I)blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
        const I cz = t / (I)nbr;
        const int b = b0 + (int)(t - cz * (I)nbr);
        const I c = cz / (I)nz;
        const int z = (int)(cz - c * (I)nz);
        const int r = srow[c];
        const int64_t dst = (((int64_t)q * nc + (int64_t)c) * nz + z) * nbp + b;
        cx<T> g{T(0), T(0)}, v{T(0), T(0)};
        if (r >= 0) {
            const int64_t src = (((int64_t)q * nsub + r) * nz + z) * nbp + b;
            g = Gs[src];
            if (q < lw) v = Ws[src];
        }
        G[dst] = g;
        if (q < lw) W[dst] = v;
    }
}

// the pixel catalog's pair count and error flags added to the galaxy catalog's
__global__ void k_merge_counters(const unsigned long long* __restrict__ from, unsigned long long* __restrict__ to)
{
    to[0] += from[0];
    to[1] |= from[1];
}

static unsigned grid_blocks(int64_t m, int n_sm)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)n_sm * 16));
}

cudaError_t launch_grid_sums(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1, const float* g2,
                             const float* w, const uint8_t* zb, int nz, long long x0, long long y0, long long pq,
                             int npx, int npy, double* scratch, int* flags, int n_sm, cudaStream_t st)
{
    const int64_t npix = (int64_t)nz * npx * npy;
    k_grid_zero<<<grid_blocks(3 * npix, n_sm), 256, 0, st>>>(3 * npix, scratch);
    if (n > 0)
        k_grid_scatter<<<grid_blocks(n, n_sm), 256, 0, st>>>(n, xq, yq, g1, g2, w, zb, nz, x0, y0, pq, npx, npy,
                                                              scratch);
    k_grid_flags<<<grid_blocks(npix, n_sm), 256, 0, st>>>(npix, scratch, flags);
    return cudaGetLastError();
}

cudaError_t launch_grid_emit(int nz, int npx, int npy, long long x0, long long y0, long long pq, const double* scratch,
                             const int* rank, int32_t* oxq, int32_t* oyq, float* og1, float* og2, float* ow,
                             uint8_t* ozb, int n_sm, cudaStream_t st)
{
    const int64_t npix = (int64_t)nz * npx * npy;
    k_grid_emit<<<grid_blocks(npix, n_sm), 256, 0, st>>>(npix, npx, npy, x0, y0, pq, scratch, rank, oxq, oyq, og1,
                                                          og2, ow, ozb);
    return cudaGetLastError();
}

cudaError_t launch_grid_combine_map(int64_t nc, const int* centre_idx, const int2* pos, const uint8_t* zs,
                                    long long x0, long long y0, long long pq, int npx, int npy, const int* flags,
                                    const int* rank, int64_t n_pix, uint8_t* pmask, int n_sm, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(pmask, 0, (size_t)n_pix, st);
    if (e != cudaSuccess) return e;
    k_grid_centre_mask<<<grid_blocks(nc, n_sm), 256, 0, st>>>(nc, centre_idx, pos, zs, x0, y0, pq, npx, npy, flags,
                                                               rank, pmask);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grid_gather(int64_t nc, int nz, int nb, int b0, int b1, int n_max, const int* centre_idx,
                               const int2* pos, const uint8_t* zs, long long x0, long long y0, long long pq, int npx,
                               int npy, const int* flags, const int* rank, int64_t nsub, const int* sub_centre_idx,
                               const int* sub_perm, int* inv, int* srow, const cx<T>* Gs, const cx<T>* Ws, cx<T>* G,
                               cx<T>* W, const unsigned long long* sub_pairs, unsigned long long* pairs, int n_sm,
                               cudaStream_t st)
{
    k_merge_counters<<<1, 1, 0, st>>>(sub_pairs, pairs);
    if (nsub > 0)
        k_grid_invert<<<grid_blocks(nsub, n_sm), 256, 0, st>>>(nsub, sub_centre_idx, sub_perm, inv);
    const int lg = 2 * n_max + 3, lw = 2 * n_max + 1;
    if (nc > 0 && b1 > b0) {
        k_grid_rows<<<grid_blocks(nc, n_sm), 256, 0, st>>>(nc, centre_idx, pos, zs, x0, y0, pq, npx, npy, flags,
                                                           rank, inv, srow);
        const int64_t ncz = nc * nz, m = ncz * (b1 - b0);
        const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 4LL * n_sm)), lg);
        if (m < 0x7fffffffLL)
            k_grid_copy<T, uint32_t><<<grid, 256, 0, st>>>((uint32_t)ncz, nz, nb_pad(nb), b0, b1 - b0, lw, srow,
                                                           nsub, Gs, Ws, G, W);
        else
            k_grid_copy<T, int64_t><<<grid, 256, 0, st>>>(ncz, nz, nb_pad(nb), b0, b1 - b0, lw, srow, nsub, Gs, Ws,
                                                          G, W);
    }
    return cudaGetLastError();
}

template cudaError_t launch_grid_gather<float>(int64_t, int, int, int, int, int, const int*, const int2*,
                                               const uint8_t*, long long, long long, long long, int, int, const int*,
                                               const int*, int64_t, const int*, const int*, int*, int*,
                                               const cx<float>*, const cx<float>*, cx<float>*, cx<float>*,
                                               const unsigned long long*, unsigned long long*, int, cudaStream_t);
template cudaError_t launch_grid_gather<double>(int64_t, int, int, int, int, int, const int*, const int2*,
                                                const uint8_t*, long long, long long, long long, int, int, const int*,
                                                const int*, int64_t, const int*, const int*, int*, int*,
                                                const cx<double>*, const cx<double>*, cx<double>*, cx<double>*,
                                                const unsigned long long*, unsigned long long*, int, cudaStream_t);

}  // namespace mp3
