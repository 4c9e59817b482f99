// Stage (b): multipole components Upsilon_{mu,n}(b1,b2) and N_n(b1,b2), sums over the centre
// galaxies of products of two moments (paper Sec. 3.1, Eqs. Upsilon0_Derivation, Upsilon1-3,
// 3PCF_Normalization, and Eq. tomoGn for tomography).
//
// SIMT form: one CTA per (Z-triplet, component, order n) group and per slice of the centre
// axis. For a tile of centres the CTA stages c_i X_i(b1) and Y_i(b2) in shared memory; each
// thread owns a few (b1, b2) outputs and accumulates the tile in T, adding tile sums in FP64.
// Slices are written to a partial buffer and summed in a fixed order, so results are
// deterministic.
#include "common.cuh"

namespace mp3 {

constexpr int kTile = 32;
constexpr int kThreads = 256;

template <typename T, int MAXO>
__global__ void __launch_bounds__(kThreads) contract_kernel(const ContractArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = a.nb, nz = a.nz, n_max = a.n_max;
    cx<T>* Xs = reinterpret_cast<cx<T>*>(smem_raw);  // [kTile][nb]
    cx<T>* Ys = Xs + kTile * nb;                      // [kTile][nb]
    const int per_zt = groups_per_zt(n_max);
    const int g = blockIdx.x, sl = blockIdx.y;
    const int zt = g / per_zt, loc = g % per_zt;
    const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
    int kind, n;
    if (loc < 4 * (n_max + 1)) {
        kind = loc / (n_max + 1);
        n = loc % (n_max + 1);
    } else {
        kind = 4;
        n = loc - 4 * (n_max + 1);
    }
    // orders and conjugations of the first (X) and second (Y) moment
    int mx, my;
    bool xconj = false, yconj = false;
    switch (kind) {
        case 0: mx = n - 3; my = -n - 3; break;                   // G_{n-3} G_{-n-3}
        case 1: mx = n - 1; my = -n - 1; break;                   // G_{n-1} G_{-n-1}
        case 2: mx = -n - 1; my = -n - 3; xconj = true; break;    // G_{-n-1}^* G_{-n-3}
        case 3: mx = n - 3; my = n - 1; yconj = true; break;      // G_{n-3} G_{n-1}^*
        default: mx = n; my = n; yconj = true; break;             // W_n W_n^*
    }
    const int off = kind < 4 ? n_max + 3 : 0;
    const int nbp = nb_pad(nb);
    const size_t plane = (size_t)a.n_centres * nz * nbp;  // stride between order slots
    const cx<T>* src = kind < 4 ? a.G : a.W;
    const int nbb = nb * nb;
    // only the centres of z-bin z1 (a contiguous range of the z-sorted centre list)
    const int zc0 = a.zrange ? a.zrange[z1] : 0, zc1 = a.zrange ? a.zrange[z1 + 1] : a.n_centres;
    const int per = (zc1 - zc0 + a.splits - 1) / a.splits;
    const int c0 = min(zc1, zc0 + sl * per);
    const int c1 = min(zc1, c0 + per);

    double accd[MAXO][2];
#pragma unroll
    for (int q = 0; q < MAXO; ++q) accd[q][0] = accd[q][1] = 0.0;

    for (int t0 = c0; t0 < c1; t0 += kTile) {
        for (int idx = threadIdx.x; idx < kTile * nb; idx += kThreads) {
            const int tt = idx / nb, b = idx % nb;
            const int c = t0 + tt;
            cx<T> X{T(0), T(0)}, Y{T(0), T(0)};
            if (c < c1) {
                const int d = a.centre_idx[c];
                const int zc = a.zs ? (int)a.zs[d] : 0;
                if (zc == z1) {
                    const Pay<T> pv = a.pay[d];
                    cx<T> coef;
                    if (kind == 4) {
                        coef = cx<T>{pv.w, T(0)};
                    } else if (kind == 1) {
                        coef = cx<T>{-pv.a, pv.b};  // -(w gamma)^*
                    } else {
                        coef = cx<T>{-pv.a, -pv.b};  // -(w gamma)
                    }
                    X = src[(size_t)(mx + off) * plane + ((size_t)c * nz + z2) * nbp + b];
                    Y = src[(size_t)(my + off) * plane + ((size_t)c * nz + z3) * nbp + b];
                    if (xconj) X = cconj(X);
                    if (yconj) Y = cconj(Y);
                    X = cmul(coef, X);
                }
            }
            Xs[tt * nb + b] = X;
            Ys[tt * nb + b] = Y;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXO; ++q) {
            const int o = threadIdx.x + q * kThreads;
            if (o < nbb) {
                const int b1 = o / nb, b2 = o % nb;
                T sr = T(0), si = T(0);
#pragma unroll 8
                for (int tt = 0; tt < kTile; ++tt) {
                    const cx<T> x = Xs[tt * nb + b1], y = Ys[tt * nb + b2];
                    sr += x.x * y.x - x.y * y.y;
                    si += x.x * y.y + x.y * y.x;
                }
                accd[q][0] += (double)sr;
                accd[q][1] += (double)si;
            }
        }
        __syncthreads();
    }
    const int groups = gridDim.x;
#pragma unroll
    for (int q = 0; q < MAXO; ++q) {
        const int o = threadIdx.x + q * kThreads;
        if (o < nbb) {
            double* dst = a.partial + 2 * (((size_t)sl * groups + g) * nbb + o);
            dst[0] = accd[q][0];
            dst[1] = accd[q][1];
        }
    }
}

__global__ void contract_reduce_kernel(const double* __restrict__ partial, int splits, int groups,
                                       int nz, int nb, int n_max, double* __restrict__ ups,
                                       double* __restrict__ norm)
{
    const int nbb = nb * nb;
    const int per_zt = groups_per_zt(n_max);
    const int64_t total = (int64_t)groups * nbb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / nbb), o = (int)(t % nbb);
        double sr = 0.0, si = 0.0;
        for (int s = 0; s < splits; ++s) {
            const double* p = partial + 2 * (((size_t)s * groups + g) * nbb + o);
            sr += p[0];
            si += p[1];
        }
        const int zt = g / per_zt, loc = g % per_zt;
        double* dst;
        if (loc < 4 * (n_max + 1)) {
            const int kind = loc / (n_max + 1), n = loc % (n_max + 1);
            dst = ups + 2 * ((((size_t)zt * 4 + kind) * (n_max + 1) + n) * nbb + o);
        } else {
            const int n = loc - 4 * (n_max + 1);
            dst = norm + 2 * (((size_t)zt * (2 * n_max + 1) + n) * nbb + o);
        }
        dst[0] += sr;
        dst[1] += si;
    }
}

// exclude_degenerate with the tensor-core forms: the b1 = b2 blocks of the Z-triplets with
// Z2 = Z3, the only blocks from which the j = k share is removed, summed again over the centres
// with the FP32 moments' products formed and accumulated in FP64. The j = k share is the largest
// part of these blocks when a bin holds few neighbours, so removing it from a split-BF16 sum would
// leave that sum's rounding of the removed share in the small remainder. Block (diagonal group,
// slice): lanes over the bins, warps over the slice's centres, a fixed-order reduction over the
// warps; the result replaces the tensor-core slice partial of the same (slice, group, b, b), so the
// slice reduction that follows adds it like any other partial.
constexpr int kDiagWarps = 8;

__global__ void __launch_bounds__(kDiagWarps * 32) contract_diag_kernel(const ContractArgs<float> a)
{
    const int nb = a.nb, nz = a.nz, n_max = a.n_max;
    const int per_zt = groups_per_zt(n_max);
    const int loc = blockIdx.x % per_zt, zz = blockIdx.x / per_zt;  // zz = z1 * nz + z2, z3 = z2
    const int z1 = zz / nz, z2 = zz % nz;
    const int zt = (z1 * nz + z2) * nz + z2;
    const int g = zt * per_zt + loc, sl = blockIdx.y;
    int kind, n;
    if (loc < 4 * (n_max + 1)) {
        kind = loc / (n_max + 1);
        n = loc % (n_max + 1);
    } else {
        kind = 4;
        n = loc - 4 * (n_max + 1);
    }
    int mx, my;
    bool xconj = false, yconj = false;
    switch (kind) {
        case 0: mx = n - 3; my = -n - 3; break;
        case 1: mx = n - 1; my = -n - 1; break;
        case 2: mx = -n - 1; my = -n - 3; xconj = true; break;
        case 3: mx = n - 3; my = n - 1; yconj = true; break;
        default: mx = n; my = n; yconj = true; break;
    }
    const int off = kind < 4 ? n_max + 3 : 0;
    const int nbp = nb_pad(nb);
    const size_t plane = (size_t)a.n_centres * nz * nbp;
    const cx<float>* src = kind < 4 ? a.G : a.W;
    const int zc0 = a.zrange ? a.zrange[z1] : 0, zc1 = a.zrange ? a.zrange[z1 + 1] : a.n_centres;
    const int per = (zc1 - zc0 + a.splits - 1) / a.splits;
    const int c0 = min(zc1, zc0 + sl * per), c1 = min(zc1, c0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[kDiagWarps][kMaxBins][2];
    for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        double sr = 0.0, si = 0.0;
        if (b < nb) {
            for (int c = c0 + warp; c < c1; c += kDiagWarps) {
                const int d = a.centre_idx[c];
                if ((a.zs ? (int)a.zs[d] : 0) != z1) continue;
                const Pay<float> pv = a.pay[d];
                cx<double> coef;
                if (kind == 4) coef = cx<double>{(double)pv.w, 0.0};
                else if (kind == 1) coef = cx<double>{-(double)pv.a, (double)pv.b};
                else coef = cx<double>{-(double)pv.a, -(double)pv.b};
                const cx<float> xf = src[(size_t)(mx + off) * plane + ((size_t)c * nz + z2) * nbp + b];
                const cx<float> yf = src[(size_t)(my + off) * plane + ((size_t)c * nz + z2) * nbp + b];
                cx<double> x{(double)xf.x, xconj ? -(double)xf.y : (double)xf.y};
                const cx<double> y{(double)yf.x, yconj ? -(double)yf.y : (double)yf.y};
                x = cmul(coef, x);
                sr += x.x * y.x - x.y * y.y;
                si += x.x * y.y + x.y * y.x;
            }
            red[warp][b][0] = sr;
            red[warp][b][1] = si;
        }
    }
    __syncthreads();
    const int groups = nz * nz * nz * per_zt, nbb = nb * nb;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < kDiagWarps; ++w) {
            tr += red[w][b][0];
            ti += red[w][b][1];
        }
        double* dst = a.partial + 2 * (((size_t)sl * groups + g) * nbb + (size_t)b * nb + b);
        dst[0] = tr;
        dst[1] = ti;
    }
}

cudaError_t launch_contract_diag(const ContractArgs<float>& a, cudaStream_t st)
{
    if (a.splits < 1 || a.n_centres <= 0) return cudaSuccess;
    dim3 grid(a.nz * a.nz * groups_per_zt(a.n_max), a.splits);
    contract_diag_kernel<<<grid, kDiagWarps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_contract_t(const ContractArgs<T>& a, cudaStream_t st)
{
    const int groups = a.nz * a.nz * a.nz * groups_per_zt(a.n_max);
    dim3 grid(groups, a.splits);
    const int nbb = a.nb * a.nb;
    const size_t smem = sizeof(cx<T>) * 2 * kTile * a.nb;
    cudaError_t e = cudaSuccess;
    if (nbb <= kThreads)
        e = set_smem_attr(contract_kernel<T, 1>, smem);
    else if (nbb <= 4 * kThreads)
        e = set_smem_attr(contract_kernel<T, 4>, smem);
    else
        e = set_smem_attr(contract_kernel<T, 16>, smem);
    if (e != cudaSuccess) return e;
    if (nbb <= kThreads)
        contract_kernel<T, 1><<<grid, kThreads, smem, st>>>(a);
    else if (nbb <= 4 * kThreads)
        contract_kernel<T, 4><<<grid, kThreads, smem, st>>>(a);
    else
        contract_kernel<T, 16><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_contract_f32(const ContractArgs<float>& a, cudaStream_t st)
{
    return launch_contract_t(a, st);
}

cudaError_t launch_contract_f64(const ContractArgs<double>& a, cudaStream_t st)
{
    return launch_contract_t(a, st);
}

cudaError_t launch_contract_reduce(const double* partial, int splits, int nz, int nb, int n_max,
                                   double* ups, double* norm, cudaStream_t st)
{
    const int groups = nz * nz * nz * groups_per_zt(n_max);
    const int64_t total = (int64_t)groups * nb * nb;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    contract_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, splits, groups, nz, nb, n_max,
                                                             ups, norm);
    return cudaGetLastError();
}

}  // namespace mp3
