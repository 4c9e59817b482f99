// FP64 stages after the contraction: the edge-correction solve (paper Sec. 3.4), the multipole
// sum to Gamma^x(phi) and its conversion to the centroid projection (Sec. 2.3, Sec. 4), and the
// aperture-measure integrals (Sec. 5.2, App. C).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace mp3 {

// ------------------------------------------------------------------ c1: edge correction

// Solves A X = B in shared memory for one system (D x D complex A, D x 4 complex B, both
// overwritten; X in B): Gaussian elimination with partial pivoting (largest |pivot|, lowest row
// on ties) by the whole block, back substitution by four warps. Returns true if a pivot was zero.
// Per elimination step: the pivot by a warp-shuffle argmax and one pass over the warps' results,
// the multipliers A_rk / A_kk once per row (stored in the finished column k), then the update.
__device__ bool block_solve4(cx<double>* A, cx<double>* B, int D, double* red_v, int* red_i, int* s_bad)
{
    const int tid = threadIdx.x, lane = tid & 31, nw = blockDim.x >> 5;
    for (int k = 0; k < D && !*s_bad; ++k) {
        double best = -1.0;
        int bi = D;
        for (int r = k + tid; r < D; r += blockDim.x) {
            const cx<double> v = A[(size_t)r * D + k];
            const double m2 = v.x * v.x + v.y * v.y;
            if (m2 > best) {
                best = m2;
                bi = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_v[tid >> 5] = best;
            red_i[tid >> 5] = bi;
        }
        __syncthreads();
        double pv = red_v[0];
        int piv = red_i[0];
        for (int w = 1; w < nw; ++w) {
            const double ov = red_v[w];
            const int oi = red_i[w];
            if (ov > pv || (ov == pv && oi < piv)) {
                pv = ov;
                piv = oi;
            }
        }
        if (!(pv > 0.0)) {
            if (tid == 0) *s_bad = 1;
            __syncthreads();
            break;
        }
        if (piv != k) {
            for (int j = k + tid; j < D; j += blockDim.x) {
                const cx<double> t = A[(size_t)k * D + j];
                A[(size_t)k * D + j] = A[(size_t)piv * D + j];
                A[(size_t)piv * D + j] = t;
            }
            for (int j = tid; j < 4; j += blockDim.x) {
                const cx<double> t = B[k * 4 + j];
                B[k * 4 + j] = B[piv * 4 + j];
                B[piv * 4 + j] = t;
            }
        }
        __syncthreads();
        const cx<double> akk = A[(size_t)k * D + k];
        for (int r = k + 1 + tid; r < D; r += blockDim.x) A[(size_t)r * D + k] = cdiv(A[(size_t)r * D + k], akk);
        __syncthreads();
        const int rows = D - k - 1, cols = D - k - 1 + 4;
        for (int idx = tid; idx < rows * cols; idx += blockDim.x) {
            const int r = k + 1 + idx / cols, jj = idx % cols;
            const cx<double> f = A[(size_t)r * D + k];
            if (jj < D - k - 1) {
                const int j = k + 1 + jj;
                A[(size_t)r * D + j] = csub(A[(size_t)r * D + j], cmul(f, A[(size_t)k * D + j]));
            } else {
                const int mu = jj - (D - k - 1);
                B[r * 4 + mu] = csub(B[r * 4 + mu], cmul(f, B[k * 4 + mu]));
            }
        }
        __syncthreads();
    }
    const bool bad = *s_bad != 0;
    const int warp = tid >> 5;
    if (!bad && warp < 4) {
        const int mu = warp;
        for (int k = D - 1; k >= 0; --k) {
            double sr = 0.0, si = 0.0;
            for (int q = k + 1 + lane; q < D; q += 32) {
                const cx<double> t = cmul(A[(size_t)k * D + q], B[q * 4 + mu]);
                sr += t.x;
                si += t.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) {
                const cx<double> rhs{B[k * 4 + mu].x - sr, B[k * 4 + mu].y - si};
                B[k * 4 + mu] = cdiv(rhs, A[(size_t)k * D + k]);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    return bad;
}

// element (l, n) of the extended mode-coupling matrix of system (zt, b1, b2): N_{l-n}, with
// N_{-m}(b1, b2) = N_m(b2, b1) of the Z2 <-> Z3 swapped triplet (App. A)
__device__ __forceinline__ cx<double> coupling(const PostArgs& p, const cx<double>* Nn, int zt, int zsw, int b1,
                                               int b2, int m)
{
    const int nb = p.nb, nmax = p.n_max, NW = 2 * nmax + 1;
    if (p.norm_truncate && (m > nmax || m < -nmax)) return cx<double>{0.0, 0.0};
    if (m >= 0) return Nn[(((size_t)zt * NW + m) * nb + b1) * nb + b2];
    return Nn[(((size_t)zsw * NW + (-m)) * nb + b2) * nb + b1];
}

// Block per (Z-triplet, b1, b2). The (2 n_max + 1)^2 complex matrix N_{l-n} and the four
// right-hand sides Upsilon_{mu,l} live in shared memory and are solved by block_solve4.
__global__ void __launch_bounds__(256) edge_correct_kernel(const PostArgs p, const double* __restrict__ ups,
                                                           const double* __restrict__ norm,
                                                           double* __restrict__ gam,
                                                           unsigned long long* nsing)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = p.n_max, D = 2 * nmax + 1, nb = p.nb, nz = p.nz;
    const int NN = nmax + 1;
    cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
    cx<double>* B = A + (size_t)D * D;
    __shared__ double red_v[256];
    __shared__ int red_i[256];
    __shared__ int s_bad;
    const int sys = blockIdx.x;
    const int b2 = sys % nb, b1 = (sys / nb) % nb, zt = sys / (nb * nb);
    const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
    const int zsw = (z1 * nz + z3) * nz + z2;
    const int tid = threadIdx.x;
    const cx<double>* U = reinterpret_cast<const cx<double>*>(ups);
    const cx<double>* Nn = reinterpret_cast<const cx<double>*>(norm);

    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int l = idx / D - nmax, nn = idx % D - nmax;
        A[idx] = coupling(p, Nn, zt, zsw, b1, b2, l - nn);
    }
    for (int idx = tid; idx < D * 4; idx += blockDim.x) {
        const int l = idx / 4 - nmax, mu = idx % 4;
        cx<double> v;
        if (l >= 0) {
            v = U[((((size_t)zt * 4 + mu) * NN + l) * nb + b1) * nb + b2];
        } else {
            const int mus = mu == 2 ? 3 : (mu == 3 ? 2 : mu);
            v = U[((((size_t)zsw * 4 + mus) * NN + (-l)) * nb + b2) * nb + b1];
        }
        B[idx] = v;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (tid == 0) {
        const cx<double> n0 = A[(size_t)nmax * D + nmax];
        if (n0.x == 0.0 && n0.y == 0.0) s_bad = 1;
    }
    __syncthreads();
    const bool bad = block_solve4(A, B, D, red_v, red_i, &s_bad);
    cx<double>* out = reinterpret_cast<cx<double>*>(gam);
    for (int idx = tid; idx < D * 4; idx += blockDim.x) {
        const int nn = idx / 4, mu = idx % 4;
        out[((((size_t)zt * 4 + mu) * D + nn) * nb + b1) * nb + b2] =
            bad ? cx<double>{nan(""), nan("")} : B[idx];
    }
    if (bad && tid == 0) atomicAdd(nsing, 1ULL);
}

// Adjoint of the solve A X = B of system (zt, b1, b2): Y = A^{-H} dL/dX (the gradient of the
// right-hand sides) and, for the matrix, dL/dA_{ln} = -sum_mu Y_mu(l) conj(X_mu(n)), summed along
// each diagonal j = l - n (A is Toeplitz in l - n). Per system the scratch holds Y [D][4] then the
// diagonal sums [2D - 1] (j = -(D-1)..D-1). Systems that were singular get zeros.
__global__ void __launch_bounds__(256) edge_correct_adjoint_kernel(const PostArgs p, const double* __restrict__ norm,
                                                                   const double* __restrict__ gam,
                                                                   const double* __restrict__ ggam,
                                                                   double* __restrict__ scratch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = p.n_max, D = 2 * nmax + 1, nb = p.nb, nz = p.nz;
    cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
    cx<double>* B = A + (size_t)D * D;
    cx<double>* X = B + (size_t)D * 4;
    __shared__ double red_v[256];
    __shared__ int red_i[256];
    __shared__ int s_bad;
    const int sys = blockIdx.x;
    const int b2 = sys % nb, b1 = (sys / nb) % nb, zt = sys / (nb * nb);
    const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
    const int zsw = (z1 * nz + z3) * nz + z2;
    const int tid = threadIdx.x;
    const cx<double>* Nn = reinterpret_cast<const cx<double>*>(norm);
    const cx<double>* Gm = reinterpret_cast<const cx<double>*>(gam);
    const cx<double>* gG = reinterpret_cast<const cx<double>*>(ggam);
    // A^H: element (l, n) = conj(A_{n l}) = conj(N_{n - l})
    for (int idx = tid; idx < D * D; idx += blockDim.x) {
        const int l = idx / D - nmax, nn = idx % D - nmax;
        A[idx] = cconj(coupling(p, Nn, zt, zsw, b1, b2, nn - l));
    }
    for (int idx = tid; idx < D * 4; idx += blockDim.x) {
        const int nn = idx / 4, mu = idx % 4;
        const size_t at = ((((size_t)zt * 4 + mu) * D + nn) * nb + b1) * nb + b2;
        B[idx] = gG[at];
        X[idx] = Gm[at];
    }
    if (tid == 0) {
        s_bad = 0;
        const cx<double> n0 = A[(size_t)nmax * D + nmax];
        if (n0.x == 0.0 && n0.y == 0.0) s_bad = 1;
        for (int i = 0; i < D * 4 && !s_bad; ++i)
            if (!(isfinite(X[i].x) && isfinite(X[i].y))) s_bad = 1;
    }
    __syncthreads();
    const bool bad = block_solve4(A, B, D, red_v, red_i, &s_bad);
    cx<double>* out = reinterpret_cast<cx<double>*>(scratch) + (size_t)sys * (D * 4 + 2 * D - 1);
    for (int idx = tid; idx < D * 4; idx += blockDim.x) out[idx] = bad ? cx<double>{0.0, 0.0} : B[idx];
    for (int j = -(D - 1) + tid; j <= D - 1; j += blockDim.x) {
        double sr = 0.0, si = 0.0;
        if (!bad) {
            const int l0 = max(0, j), l1 = min(D - 1, D - 1 + j);
            for (int l = l0; l <= l1; ++l) {
                const int nn = l - j;
                for (int mu = 0; mu < 4; ++mu) {
                    const cx<double> t = cmul(B[l * 4 + mu], cconj(X[nn * 4 + mu]));
                    sr -= t.x;
                    si -= t.y;
                }
            }
        }
        out[D * 4 + (j + D - 1)] = cx<double>{sr, si};
    }
}

// dL/dUpsilon [z3][4][n_max+1][nb][nb] and dL/dN [z3][2n_max+1][nb][nb] from the per-system
// scratch: each stored element is read by its own system and, for orders >= 1, by the system of
// the swapped triplet and transposed bins through the App. A symmetries.
__global__ void edge_correct_adjoint_gather(const PostArgs p, const double* __restrict__ scratch,
                                            double* __restrict__ gups, double* __restrict__ gnorm)
{
    const int nmax = p.n_max, D = 2 * nmax + 1, nb = p.nb, nz = p.nz, NN = nmax + 1, NW = 2 * nmax + 1;
    const int z3 = nz * nz * nz;
    const int per = D * 4 + 2 * D - 1;
    const cx<double>* S = reinterpret_cast<const cx<double>*>(scratch);
    const int64_t nu = (int64_t)z3 * 4 * NN * nb * nb, nn_ = (int64_t)z3 * NW * nb * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nu + nn_;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nu) {
            const int b2 = (int)(t % nb), b1 = (int)((t / nb) % nb);
            const int l = (int)((t / ((int64_t)nb * nb)) % NN);
            const int mu = (int)((t / ((int64_t)nb * nb * NN)) % 4);
            const int zt = (int)(t / ((int64_t)nb * nb * NN * 4));
            const int z1 = zt / (nz * nz), zb = (zt / nz) % nz, zc = zt % nz;
            const int zsw = (z1 * nz + zc) * nz + zb;
            const int mus = mu == 2 ? 3 : (mu == 3 ? 2 : mu);
            cx<double> v = S[((size_t)(zt * nb + b1) * nb + b2) * per + (l + nmax) * 4 + mu];
            if (l >= 1) v = cadd(v, S[((size_t)(zsw * nb + b2) * nb + b1) * per + (-l + nmax) * 4 + mus]);
            reinterpret_cast<cx<double>*>(gups)[t] = v;
        } else {
            const int64_t u = t - nu;
            const int b2 = (int)(u % nb), b1 = (int)((u / nb) % nb);
            const int m = (int)((u / ((int64_t)nb * nb)) % NW);
            const int zt = (int)(u / ((int64_t)nb * nb * NW));
            const int z1 = zt / (nz * nz), zb = (zt / nz) % nz, zc = zt % nz;
            const int zsw = (z1 * nz + zc) * nz + zb;
            cx<double> v{0.0, 0.0};
            if (!(p.norm_truncate && m > nmax)) {
                v = S[((size_t)(zt * nb + b1) * nb + b2) * per + D * 4 + (m + D - 1)];
                if (m >= 1) v = cadd(v, S[((size_t)(zsw * nb + b2) * nb + b1) * per + D * 4 + (-m + D - 1)]);
            }
            reinterpret_cast<cx<double>*>(gnorm)[u] = v;
        }
    }
}

cudaError_t launch_edge_correct_adjoint(const PostArgs& p, const double* norm, const double* gam,
                                        const double* ggam, double* scratch, double* gups, double* gnorm,
                                        cudaStream_t st)
{
    const int D = 2 * p.n_max + 1;
    const size_t smem = sizeof(cx<double>) * ((size_t)D * D + (size_t)D * 8);
    cudaError_t e = set_smem_attr(edge_correct_adjoint_kernel, smem);
    if (e != cudaSuccess) return e;
    const int systems = p.nz * p.nz * p.nz * p.nb * p.nb;
    edge_correct_adjoint_kernel<<<systems, 256, smem, st>>>(p, norm, gam, ggam, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)p.nz * p.nz * p.nz * p.nb * p.nb * (4 * (p.n_max + 1) + 2 * p.n_max + 1);
    edge_correct_adjoint_gather<<<(unsigned)std::min<int64_t>((total + 255) / 256, 65535), 256, 0, st>>>(
        p, scratch, gups, gnorm);
    return cudaGetLastError();
}

size_t edge_correct_adjoint_scratch(const PostArgs& p)
{
    const int D = 2 * p.n_max + 1;
    return sizeof(cx<double>) * (size_t)p.nz * p.nz * p.nz * p.nb * p.nb * (D * 4 + 2 * D - 1);
}

cudaError_t launch_edge_correct(const PostArgs& p, const double* ups, const double* norm,
                                double* gam, unsigned long long* nsing, cudaStream_t st)
{
    const int D = 2 * p.n_max + 1;
    const size_t smem = sizeof(cx<double>) * ((size_t)D * D + (size_t)D * 4);
    cudaError_t e = set_smem_attr(edge_correct_kernel, smem);
    if (e != cudaSuccess) return e;
    const int systems = p.nz * p.nz * p.nz * p.nb * p.nb;
    edge_correct_kernel<<<systems, 256, smem, st>>>(p, ups, norm, gam, nsing);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ c2: to_gamma

// rotation factor taking Gamma^x_mu to Gamma^cen_mu at (t1, t2, phi), e = e^{i phi}
__device__ __forceinline__ cx<double> centroid_factor(int mu, double t1, double t2, cx<double> e)
{
    const cx<double> ec = cconj(e);
    const cx<double> r1 = cdiv(cx<double>{t1 + t2 * ec.x, t2 * ec.y}, cx<double>{t1 + t2 * e.x, t2 * e.y});
    const cx<double> r2 = cdiv(cx<double>{t2 * ec.x - 2.0 * t1, t2 * ec.y},
                               cx<double>{t2 * e.x - 2.0 * t1, t2 * e.y});
    const cx<double> r3 = cdiv(cx<double>{t1 - 2.0 * t2 * ec.x, -2.0 * t2 * ec.y},
                               cx<double>{t1 - 2.0 * t2 * e.x, -2.0 * t2 * e.y});
    const cx<double> e2 = cmul(e, e), e3 = cmul(e2, e);
    switch (mu) {
        case 0: return cmul(cmul(cmul(r1, r2), r3), e3);
        case 1: return cmul(cdiv(cmul(r2, r3), r1), e);
        case 2: return cmul(cdiv(cmul(r1, r3), r2), e3);
        default: return cmul(cdiv(cmul(r1, r2), r3), ec);
    }
}

__global__ void to_gamma_kernel(const PostArgs p, const double* __restrict__ gam, int proj,
                                double* __restrict__ out)
{
    const int nb = p.nb, nmax = p.n_max, D = 2 * nmax + 1, np = p.n_phi;
    const int z3 = p.nz * p.nz * p.nz;
    const int64_t total = (int64_t)z3 * 4 * nb * nb * np;
    const cx<double>* G = reinterpret_cast<const cx<double>*>(gam);
    cx<double>* O = reinterpret_cast<cx<double>*>(out);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % np);
        const int64_t rest = t / np;
        const int b2 = (int)(rest % nb), b1 = (int)((rest / nb) % nb);
        const int64_t zm = rest / ((int64_t)nb * nb);  // zt * 4 + mu
        double s, c;
        sincospi((2.0 * k + 1.0) / np, &s, &c);
        const cx<double> e1{c, s};
        const size_t stride = (size_t)nb * nb;
        const cx<double>* g0 = G + (size_t)zm * D * stride + (size_t)b1 * nb + b2;
        cx<double> acc = g0[(size_t)nmax * stride];
        cx<double> ep{1.0, 0.0};
        for (int n = 1; n <= nmax; ++n) {
            ep = cmul(ep, e1);
            cx<double> t = cadd(cmul(g0[(size_t)(nmax + n) * stride], ep),
                                cmul(g0[(size_t)(nmax - n) * stride], cconj(ep)));
            // projection 2: the average of e^{i n phi} over the angular bin is e^{i n phi_k}
            // sinc(n pi / n_phi)
            if (proj == 2) t = cscale(t, sinpi((double)n / np) / (M_PI * (double)n / np));
            acc = cadd(acc, t);
        }
        if (proj == 1) acc = cmul(acc, centroid_factor((int)(zm % 4), p.nodes[b1], p.nodes[b2], e1));
        O[t] = acc;
    }
}

cudaError_t launch_to_gamma(const PostArgs& p, const double* gam, int projection, double* out,
                            cudaStream_t st)
{
    const int64_t total = (int64_t)p.nz * p.nz * p.nz * 4 * p.nb * p.nb * p.n_phi;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    to_gamma_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, gam, projection, out);
    return cudaGetLastError();
}

// Adjoint of to_gamma: dL/dGamma_n = sum_k dL/dGamma(phi_k) conj(R(phi_k)) e^{-i n phi_k}, with
// R the centroid factor (projection 1) or 1. Block per (Z-triplet, mu, b1, b2): the n_phi weighted
// gradients h_k = dL/dGamma(phi_k) conj(R(phi_k)) are formed once in shared memory, then a thread
// per n sums h_k e^{-i n phi_k} over k (the same order of terms as a direct sum); overwrites.
constexpr int kTgaThreads = 128;

__global__ void __launch_bounds__(kTgaThreads) to_gamma_adjoint_kernel(const PostArgs p,
                                                                      const double* __restrict__ gphi, int proj,
                                                                      double* __restrict__ ggam)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<double>* h = reinterpret_cast<cx<double>*>(smem_raw);  // [n_phi]
    const int nb = p.nb, nmax = p.n_max, D = 2 * nmax + 1, np = p.n_phi;
    const int64_t sys = blockIdx.x;  // ((zt * 4 + mu) * nb + b1) * nb + b2
    const int b2 = (int)(sys % nb), b1 = (int)((sys / nb) % nb);
    const int64_t zm = sys / ((int64_t)nb * nb);  // zt * 4 + mu
    const cx<double>* g = reinterpret_cast<const cx<double>*>(gphi) + sys * np;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        cx<double> v = g[k];
        if (proj) {
            double s, c;
            sincospi((2.0 * k + 1.0) / np, &s, &c);
            v = cmul(v, cconj(centroid_factor((int)(zm % 4), p.nodes[b1], p.nodes[b2], cx<double>{c, s})));
        }
        h[k] = v;
    }
    __syncthreads();
    cx<double>* O = reinterpret_cast<cx<double>*>(ggam);
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const int nn = i - nmax;
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < np; ++k) {
            double sn, cn;
            sincospi((double)nn * (2.0 * k + 1.0) / np, &sn, &cn);
            const cx<double> v = cmul(h[k], cx<double>{cn, -sn});  // e^{-i n phi_k}
            sr += v.x;
            si += v.y;
        }
        O[((size_t)zm * D + i) * nb * nb + (size_t)b1 * nb + b2] = cx<double>{sr, si};
    }
}

cudaError_t launch_to_gamma_adjoint(const PostArgs& p, const double* gphi, int projection, double* ggam,
                                    cudaStream_t st)
{
    const int64_t systems = (int64_t)p.nz * p.nz * p.nz * 4 * p.nb * p.nb;
    if (systems < 1) return cudaSuccess;
    const size_t smem = sizeof(cx<double>) * (size_t)p.n_phi;
    cudaError_t e = set_smem_attr(to_gamma_adjoint_kernel, smem);
    if (e != cudaSuccess) return e;
    to_gamma_adjoint_kernel<<<(unsigned)systems, kTgaThreads, smem, st>>>(p, gphi, projection, ggam);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ c3: to_map3

// The four filters. F_0 as printed in App. C. For mu = 1..3 (conjugate at vertex mu) the
// printed F_1 expression is evaluated with its three vertex labels rotated by
// s = (mu + 1) mod 3: with the q-vectors of Eq. QvecDef the printed expression is the kernel of
// the correlator conjugated at vertex 2 (derived from Eqs. MapGamma, CrittendenQ and the
// centroid projection), so rotating by s moves its special vertex onto vertex mu.
__device__ cx<double> aperture_filter(int mu, double t1, double t2, cx<double> e, const double th[3])
{
    const cx<double> v1{t1, 0.0}, v2{t2 * e.x, t2 * e.y};
    cx<double> q[3];
    q[0] = cx<double>{-(v1.x + v2.x) / 3.0, -(v1.y + v2.y) / 3.0};
    q[1] = cx<double>{(2.0 * v1.x - v2.x) / 3.0, (2.0 * v1.y - v2.y) / 3.0};
    q[2] = cx<double>{(2.0 * v2.x - v1.x) / 3.0, (2.0 * v2.y - v1.y) / 3.0};
    double s2[3], qq[3];
    for (int i = 0; i < 3; ++i) {
        s2[i] = th[i] * th[i];
        qq[i] = q[i].x * q[i].x + q[i].y * q[i].y;
    }
    const double T4 = (s2[0] * s2[1] + s2[0] * s2[2] + s2[1] * s2[2]) / 3.0;
    const double T2 = sqrt(T4), T6 = T2 * T4;
    const double Mfac = (s2[0] * s2[1] * s2[2] / T6) * t1 * t2 / (2.0 * M_PI * T4);
    double Z = 0.0;
    cx<double> f[3], gg[3];
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        Z += (-s2[i] + 2.0 * s2[i1] + 2.0 * s2[i2]) * qq[i];
        const cx<double> r = cscale(cmul(cconj(q[i]), csub(q[i1], q[i2])), 1.0 / qq[i]);
        f[i] = cx<double>{(s2[i1] + s2[i2]) / (2.0 * T2) + r.x * (s2[i1] - s2[i2]) / (6.0 * T2),
                          r.y * (s2[i1] - s2[i2]) / (6.0 * T2)};
        gg[i] = cx<double>{s2[i1] * s2[i2] / T4 + r.x * s2[i] * (s2[i2] - s2[i1]) / (3.0 * T4),
                           r.y * s2[i] * (s2[i2] - s2[i1]) / (3.0 * T4)};
    }
    Z /= 6.0 * T4;
    const double aq = qq[0] * qq[1] * qq[2];
    const double ez = exp(-Z);
    if (mu == 0) {
        cx<double> pr{1.0, 0.0};
        for (int i = 0; i < 3; ++i) {
            const cx<double> fc = cconj(f[i]);
            pr = cmul(pr, cmul(fc, fc));
        }
        return cscale(pr, Mfac / 24.0 * aq / T6 * ez);
    }
    const int s = (mu + 1) % 3;
    const int u1 = s, u2 = (s + 1) % 3, u3 = (s + 2) % 3;
    const cx<double> Q1 = q[u1], Q2c = cconj(q[u2]), Q3 = q[u3];
    const cx<double> F1c = cconj(f[u1]), F2 = f[u2], F3c = cconj(f[u3]), G2c = cconj(gg[u2]);
    const cx<double> q31 = cmul(Q3, Q1), q2c2 = cmul(Q2c, Q2c);
    const cx<double> f31 = cmul(F3c, F1c);
    // term 1: |q1|^2|q2|^2|q3|^2 / (24 Theta^6) f3*^2 f1*^2 f2^2
    cx<double> t = cscale(cmul(cmul(f31, f31), cmul(F2, F2)), aq / (24.0 * T6));
    // term 2: -(1/9) q3 q1 q2*^2 / Theta^4 f3* f1* f2 g2*
    t = csub(t, cscale(cmul(cmul(q31, q2c2), cmul(cmul(f31, F2), G2c)), 1.0 / (9.0 * T4)));
    // term 3: (1/27) [q3^2 q1^2 q2*^4 / (|q1|^2|q2|^2|q3|^2 Theta^2) g2*^2
    //                 + 2 theta3^2 theta1^2 / Theta^4  q3 q1 q2*^2 / (|q2|^2 Theta^2) f3* f1*]
    const cx<double> a1 = cscale(cmul(cmul(cmul(q31, q31), cmul(q2c2, q2c2)), cmul(G2c, G2c)), 1.0 / (aq * T2));
    const cx<double> a2 = cscale(cmul(cmul(q31, q2c2), f31), 2.0 * s2[u3] * s2[u1] / (T4 * qq[u2] * T2));
    t = cadd(t, cscale(cadd(a1, a2), 1.0 / 27.0));
    return cscale(t, Mfac * ez);
}

constexpr int kM3Threads = 256;

__global__ void __launch_bounds__(kM3Threads) map3_partial_kernel(const PostArgs p, const double* __restrict__ gcen,
                                                                  int n_ap, const double* __restrict__ theta,
                                                                  double* __restrict__ partial, int chunks)
{
    const int nb = p.nb, np = p.n_phi;
    const int job = blockIdx.x;  // zt * n_ap + ap
    const int zt = job / n_ap, ap = job % n_ap;
    const int64_t npts = (int64_t)4 * nb * nb * np;
    const int64_t per = (npts + chunks - 1) / chunks;
    const int64_t p0 = blockIdx.y * per, p1 = min(npts, p0 + per);
    const double th[3] = {theta[3 * ap], theta[3 * ap + 1], theta[3 * ap + 2]};
    const double dphi = 2.0 * M_PI / np;
    const cx<double>* gc = reinterpret_cast<const cx<double>*>(gcen) + (size_t)zt * npts;
    double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int64_t t = p0 + threadIdx.x; t < p1; t += blockDim.x) {
        const int k = (int)(t % np);
        const int64_t rest = t / np;
        const int b2 = (int)(rest % nb), b1 = (int)((rest / nb) % nb), mu = (int)(rest / ((int64_t)nb * nb));
        double s, c;
        sincospi((2.0 * k + 1.0) / np, &s, &c);
        const double t1 = p.nodes[b1], t2 = p.nodes[b2];
        const double w = (p.edges[b1 + 1] - p.edges[b1]) * (p.edges[b2 + 1] - p.edges[b2]) * dphi;
        const cx<double> v = cmul(gc[t], aperture_filter(mu, t1, t2, cx<double>{c, s}, th));
        for (int q = 0; q < 4; ++q)
            if (q == mu) {
                acc[q][0] += v.x * w;
                acc[q][1] += v.y * w;
            }
    }
    __shared__ double red[kM3Threads / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q)
        for (int r = 0; r < 2; ++r) {
            double v = acc[q][r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][2 * q + r] = v;
        }
    __syncthreads();
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int wi = 0; wi < kM3Threads / 32; ++wi) v += red[wi][threadIdx.x];
        partial[((size_t)job * chunks + blockIdx.y) * 8 + threadIdx.x] = v;
    }
}

__global__ void map3_final_kernel(int jobs, int chunks, const double* __restrict__ partial,
                                  double* __restrict__ corr, double* __restrict__ m8)
{
    const int job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= jobs) return;
    double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ch = 0; ch < chunks; ++ch)
        for (int q = 0; q < 8; ++q) c[q] += partial[((size_t)job * chunks + ch) * 8 + q];
    if (corr)
        for (int q = 0; q < 8; ++q) corr[(size_t)job * 8 + q] = c[q];
    if (m8) {
        // c0 = <M^3>, c1 = <M* M^2>, c2 = <M M* M>, c3 = <M^2 M*>; Eqs. MapTrafo8_1-8
        const double r0 = c[0], i0 = c[1], r1 = c[2], i1 = c[3], r2 = c[4], i2 = c[5], r3 = c[6], i3 = c[7];
        double* o = m8 + (size_t)job * 8;
        o[0] = (r3 + r2 + r1 + r0) / 4.0;
        o[1] = (i3 + i2 - i1 + i0) / 4.0;
        o[2] = (i3 - i2 + i1 + i0) / 4.0;
        o[3] = (-i3 + i2 + i1 + i0) / 4.0;
        o[4] = (r3 + r2 - r1 - r0) / 4.0;
        o[5] = (r3 - r2 + r1 - r0) / 4.0;
        o[6] = (-r3 + r2 + r1 - r0) / 4.0;
        o[7] = (i3 + i2 + i1 - i0) / 4.0;
    }
}

// Adjoint of the aperture measures: the correlators are c_mu = sum gcen_mu F_mu w (w = the
// d theta1 d theta2 d phi weights) and m8 = L c (Eqs. MapTrafo8_1-8, a real linear map of the
// real and imaginary parts). With dL/dc = L^T dL/dm8 (+ dL/dcorr), dL/dgcen_mu =
// sum_apertures dL/dc_mu conj(F_mu) w. Thread per gcen element; overwrites.
__device__ __forceinline__ void map3_corr_grad(const double* gm8, const double* gcorr, size_t job, double g[8])
{
    for (int q = 0; q < 8; ++q) g[q] = gcorr ? gcorr[job * 8 + q] : 0.0;
    if (gm8) {
        const double* o = gm8 + job * 8;
        // transpose of the combination in map3_final_kernel; g = (r0, i0, r1, i1, r2, i2, r3, i3)
        g[0] += (o[0] - o[4] - o[5] - o[6]) / 4.0;
        g[2] += (o[0] - o[4] + o[5] + o[6]) / 4.0;
        g[4] += (o[0] + o[4] - o[5] + o[6]) / 4.0;
        g[6] += (o[0] + o[4] + o[5] - o[6]) / 4.0;
        g[1] += (o[1] + o[2] + o[3] - o[7]) / 4.0;
        g[3] += (-o[1] + o[2] + o[3] + o[7]) / 4.0;
        g[5] += (o[1] - o[2] + o[3] + o[7]) / 4.0;
        g[7] += (o[1] + o[2] - o[3] + o[7]) / 4.0;
    }
}

__global__ void map3_adjoint_kernel(const PostArgs p, int n_ap, const double* __restrict__ theta,
                                    const double* __restrict__ gcorr, const double* __restrict__ gm8,
                                    double* __restrict__ ggcen)
{
    const int nb = p.nb, np = p.n_phi;
    const int64_t npts = (int64_t)4 * nb * nb * np;
    const int64_t total = (int64_t)p.nz * p.nz * p.nz * npts;
    const double dphi = 2.0 * M_PI / np;
    cx<double>* O = reinterpret_cast<cx<double>*>(ggcen);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t zt = t / npts, r = t % npts;
        const int k = (int)(r % np);
        const int64_t rest = r / np;
        const int b2 = (int)(rest % nb), b1 = (int)((rest / nb) % nb), mu = (int)(rest / ((int64_t)nb * nb));
        double s, c;
        sincospi((2.0 * k + 1.0) / np, &s, &c);
        const double t1 = p.nodes[b1], t2 = p.nodes[b2];
        const double w = (p.edges[b1 + 1] - p.edges[b1]) * (p.edges[b2 + 1] - p.edges[b2]) * dphi;
        cx<double> acc{0.0, 0.0};
        for (int ap = 0; ap < n_ap; ++ap) {
            double g[8];
            map3_corr_grad(gm8, gcorr, (size_t)zt * n_ap + ap, g);
            const double th[3] = {theta[3 * ap], theta[3 * ap + 1], theta[3 * ap + 2]};
            const cx<double> F = aperture_filter(mu, t1, t2, cx<double>{c, s}, th);
            acc = cadd(acc, cscale(cmul(cx<double>{g[2 * mu], g[2 * mu + 1]}, cconj(F)), w));
        }
        O[t] = acc;
    }
}

cudaError_t launch_to_map3_adjoint(const PostArgs& p, int n_ap, const double* theta, const double* gcorr,
                                   const double* gm8, double* ggcen, cudaStream_t st)
{
    const int64_t total = (int64_t)p.nz * p.nz * p.nz * 4 * p.nb * p.nb * p.n_phi;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    map3_adjoint_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n_ap, theta, gcorr, gm8, ggcen);
    return cudaGetLastError();
}

// ---- the four-equation form (App. C, Eqs. MapTrafo4_1-4). The printed equations put the
// conjugate of each one-conjugate correlator on the last radius of its ordering (the convention of
// the paper's reference for these forms); the library's Gamma_1 / F_1 correlator <M^* M^2>
// conjugates the first, so A123, A132, A231 are <M^* M^2> at (t3, t1, t2), (t2, t1, t3) and
// (t1, t2, t3); <M^3>(t1, t2, t3) comes with the last.
__global__ void map3_orderings_kernel(int n_ap, const double* __restrict__ theta, double* __restrict__ theta3)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_ap) return;
    const double t1 = theta[3 * a], t2 = theta[3 * a + 1], t3 = theta[3 * a + 2];
    double* o = theta3 + 9 * a;
    o[0] = t3; o[1] = t1; o[2] = t2;
    o[3] = t2; o[4] = t1; o[5] = t3;
    o[6] = t1; o[7] = t2; o[8] = t3;
}

__global__ void map3_four_kernel(int jobs, const double* __restrict__ corr3, double* __restrict__ m4)
{
    const int job = blockIdx.x * blockDim.x + threadIdx.x;  // (Z-triplet, aperture)
    if (job >= jobs) return;
    const double* c = corr3 + (size_t)job * 3 * 8;  // [ordering][mu][re, im]
    const double a1r = c[2], a1i = c[3], a2r = c[8 + 2], a2i = c[8 + 3], a3r = c[16 + 2], a3i = c[16 + 3];
    const double mr = c[16], mi = c[17];
    double* o = m4 + (size_t)job * 4;
    o[0] = (a1r + a2r + a3r + mr) / 4.0;
    o[1] = (-a1i + a2i + a3i + mi) / 4.0;
    o[2] = (a1r + a2r - a3r - mr) / 4.0;
    o[3] = (a1i + a2i + a3i - mi) / 4.0;
}

cudaError_t launch_to_map3_four(const PostArgs& p, const double* gcen, int n_ap, const double* theta, double* theta3,
                                double* corr3, double* partial, int chunks, double* m4, cudaStream_t st)
{
    map3_orderings_kernel<<<(n_ap + 127) / 128, 128, 0, st>>>(n_ap, theta, theta3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_to_map3(p, gcen, 3 * n_ap, theta3, partial, chunks, corr3, nullptr, st);
    if (e != cudaSuccess) return e;
    const int jobs = p.nz * p.nz * p.nz * n_ap;
    map3_four_kernel<<<(jobs + 127) / 128, 128, 0, st>>>(jobs, corr3, m4);
    return cudaGetLastError();
}

cudaError_t launch_to_map3(const PostArgs& p, const double* gcen, int n_ap, const double* theta,
                           double* partial, int chunks, double* corr, double* m8, cudaStream_t st)
{
    const int jobs = p.nz * p.nz * p.nz * n_ap;
    dim3 grid(jobs, chunks);
    map3_partial_kernel<<<grid, kM3Threads, 0, st>>>(p, gcen, n_ap, theta, partial, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    map3_final_kernel<<<(jobs + 127) / 128, 128, 0, st>>>(jobs, chunks, partial, corr, m8);
    return cudaGetLastError();
}

}  // namespace mp3
