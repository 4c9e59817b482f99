// The direct estimator of the third-order aperture mass (paper Sec. 5.3, Eq. MapDirectEstimator),
// an estimate independent of the 3PCF route: at an aperture centre c and radii (t1, t2, t3),
//   num = sum over distinct i, j, k of w_i w_j w_k Q_t1(r_i) Q_t2(r_j) Q_t3(r_k) gt_i gt_j gt_k,
//   den = the same sum without the tangential shears,
// with r_i = |x_i - c|, gt_i the tangential shear about c (gt = -Re(gamma e^{-2 i zeta}), zeta the
// polar angle of x_i - c, Eq. gammatx_def) and Q the filter of Eq. CrittendenQ,
// Q_t(r) = r^2 / (4 pi t^4) exp(-r^2 / (2 t^2)); galaxies farther than rcut from c are left out
// (the paper keeps galaxies within 4 max(t)). The sums over distinct triplets follow from seven
// sums per aperture by inclusion-exclusion over the coincidences i = j, i = k, j = k: with
// A = sum a_i, AB = sum a_i b_i, ABC = sum a_i b_i c_i (a, b, c the factors of the three slots),
//   sum_{i, j, k distinct} a_i b_j c_k = A B C - AB C - AC B - BC A + 2 ABC,
// so each aperture costs one pass over the catalog. Block per (aperture, radii triple), threads
// over the galaxies, FP64 sums reduced over the block.
#include <math.h>

#include "common.cuh"

namespace mp3 {

constexpr int kDirThreads = 256;

__global__ void __launch_bounds__(kDirThreads) map3_direct_kernel(int64_t n, const int32_t* __restrict__ xq,
                                                                  const int32_t* __restrict__ yq,
                                                                  const float* __restrict__ g1,
                                                                  const float* __restrict__ g2,
                                                                  const float* __restrict__ w, double quantum,
                                                                  int n_ap, const double* __restrict__ centres,
                                                                  const double* __restrict__ theta,
                                                                  double rcut_factor, double* __restrict__ out)
{
    __shared__ double red[14][kDirThreads / 32];
    const int64_t job = blockIdx.x;  // centre * n_ap + radii triple
    const int64_t t = job / n_ap;
    const int a = (int)(job % n_ap);
    const double cx = centres[2 * t], cy = centres[2 * t + 1];
    double th[3], inv2[3], nrm[3];
    for (int l = 0; l < 3; ++l) {
        th[l] = theta[3 * a + l];
        inv2[l] = 1.0 / (2.0 * th[l] * th[l]);
        nrm[l] = 1.0 / (4.0 * M_PI * th[l] * th[l] * th[l] * th[l]);
    }
    const double rcut = rcut_factor * fmax(th[0], fmax(th[1], th[2]));
    double s[14];
#pragma unroll
    for (int v = 0; v < 14; ++v) s[v] = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double dx = (double)xq[i] * quantum - cx, dy = (double)yq[i] * quantum - cy;
        const double r2 = dx * dx + dy * dy;
        if (r2 == 0.0 || sqrt(r2) > rcut) continue;
        // tangential shear about c: -Re((g1 + i g2) (dx - i dy)^2 / r^2)
        const double gt = -((double)g1[i] * (dx * dx - dy * dy) + 2.0 * (double)g2[i] * dx * dy) / r2;
        double b[3], c[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            b[l] = (double)w[i] * r2 * nrm[l] * exp(-r2 * inv2[l]);  // w Q_tl(r)
            c[l] = b[l] * gt;
        }
        s[0] += c[0];
        s[1] += c[1];
        s[2] += c[2];
        s[3] += c[0] * c[1];
        s[4] += c[0] * c[2];
        s[5] += c[1] * c[2];
        s[6] += c[0] * c[1] * c[2];
        s[7] += b[0];
        s[8] += b[1];
        s[9] += b[2];
        s[10] += b[0] * b[1];
        s[11] += b[0] * b[2];
        s[12] += b[1] * b[2];
        s[13] += b[0] * b[1] * b[2];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < 14; ++v) {
        double x = s[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[v][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double q[14];
        for (int v = 0; v < 14; ++v) {
            q[v] = 0.0;
            for (int k = 0; k < kDirThreads / 32; ++k) q[v] += red[v][k];
        }
        out[2 * job] = q[0] * q[1] * q[2] - q[3] * q[2] - q[4] * q[1] - q[5] * q[0] + 2.0 * q[6];
        out[2 * job + 1] = q[7] * q[8] * q[9] - q[10] * q[9] - q[11] * q[8] - q[12] * q[7] + 2.0 * q[13];
    }
}

cudaError_t launch_map3_direct(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1, const float* g2,
                               const float* w, double quantum, int64_t n_cen, const double* centres, int n_ap,
                               const double* theta, double rcut_factor, double* out, cudaStream_t st)
{
    const int64_t jobs = n_cen * (int64_t)n_ap;
    if (jobs < 1) return cudaSuccess;
    if (jobs > 0x7fffffffLL) return cudaErrorInvalidValue;
    map3_direct_kernel<<<(unsigned)jobs, kDirThreads, 0, st>>>(n, xq, yq, g1, g2, w, quantum, n_ap, centres, theta,
                                                               rcut_factor, out);
    return cudaGetLastError();
}

}  // namespace mp3
