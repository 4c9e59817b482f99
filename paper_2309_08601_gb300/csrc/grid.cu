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

}  // namespace mp3
