// Shared device/host definitions of the mp3pcf CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mp3pcf.h"

namespace mp3 {

constexpr int kMaxBins = 64;   // radial bins supported by the device kernels
constexpr int kMaxNmax = 50;   // largest multipole order
constexpr int kMaxNz = 8;      // tomographic bins
constexpr int kMaxRows = 480;  // cell rows an annulus may span (host picks the cell side)

// ------------------------------------------------------------------ complex helpers

template <typename T>
struct cx {
    T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T>
__host__ __device__ __forceinline__ cx<T> cconj(cx<T> a)
{
    return {a.x, -a.y};
}

template <typename T>
__host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b)
{
    return {a.x + b.x, a.y + b.y};
}

template <typename T>
__host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b)
{
    return {a.x - b.x, a.y - b.y};
}

template <typename T>
__host__ __device__ __forceinline__ cx<T> cscale(cx<T> a, T s)
{
    return {a.x * s, a.y * s};
}

__host__ __device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b)
{
    // (a b*) / |b|^2 with a scaling step against overflow
    const double s = fabs(b.x) > fabs(b.y) ? fabs(b.x) : fabs(b.y);
    const double bx = b.x / s, by = b.y / s;
    const double d = bx * bx + by * by;
    return {(a.x * bx + a.y * by) / (d * s), (a.y * bx - a.x * by) / (d * s)};
}

// per-galaxy payload in sorted order, one aligned record: w gamma_1, w gamma_2, w
template <typename T>
struct alignas(4 * sizeof(T)) Pay {
    T a, b, w, pad;
};

// ------------------------------------------------------------------ geometry of the cell grid

struct GridDesc {
    int64_t x0, y0;     // fixed-point origin of cell (0, 0)
    int32_t side;       // cell side in fixed-point units
    int32_t ncx, ncy;   // cells per row / rows
    int32_t ncells;     // ncx * ncy (per tomographic bin)
};

// ------------------------------------------------------------------ stage (a) arguments

template <typename T>
struct MomentArgs {
    int32_t n_centres;
    const int32_t* centre_idx;  // sorted position of each centre
    const int2* pos;            // sorted fixed-point positions
    const Pay<T>* pay;          // sorted (w gamma_1, w gamma_2, w)
    const int32_t* cell_start;  // [n_z * ncells + 1], key = zbin * ncells + cy * ncx + cx
    GridDesc g;
    int32_t nz, nb, n_max;      // nb: the radial bins computed, a range [b_lo, b_lo + nb) of the layout's
    int32_t nbp;                // bins per row of the layout (nb_pad of all its bins)
    const long long* e2q;       // [nb + 1] exact squared edges in fixed-point units^2, from bin b_lo
    cx<T>* G;                   // [2 n_max + 3][n_centres][nz][nbp], offset to bin b_lo
    cx<T>* W;                   // [2 n_max + 1][n_centres][nz][nbp], offset to bin b_lo
    unsigned long long* pairs;  // [0] pair counter, [1] error flags (1: a bounded wait gave up)
    unsigned long long* queue;  // centres claimed beyond the first gridDim.x (zero at launch)
};

// launchers implemented in moments_f32.cu / moments_f64.cu
cudaError_t launch_moments_f32(const MomentArgs<float>& a, int n_sm, cudaStream_t st);
cudaError_t launch_moments_f64(const MomentArgs<double>& a, int n_sm, cudaStream_t st);

// ------------------------------------------------------------------ stage (b)

template <typename T>
struct ContractArgs {
    const cx<T>* G;
    const cx<T>* W;
    const Pay<T>* pay;         // sorted (w gamma_1, w gamma_2, w)
    const uint8_t* zs;         // sorted zbin
    const int32_t* centre_idx; // sorted position of each centre (row order of G, W)
    int32_t n_centres;
    int32_t nz, nb, n_max;
    int32_t splits;
    double* partial;  // [splits][groups][nb*nb][2]
    // device [nz + 1]: the centres of z-bin z are [zrange[z], zrange[z + 1]) of the centre list
    // (sorted by z-bin); nullptr: every centre (one z-bin)
    const int32_t* zrange;
};

cudaError_t launch_contract_f32(const ContractArgs<float>& a, cudaStream_t st);
cudaError_t launch_contract_f64(const ContractArgs<double>& a, cudaStream_t st);
// tensor-core form (FP32 moments, BF16 or TF32 hi+lo split products); plan_only computes the
// number of centre slices (*splits) without launching; coef is scratch for n_centres float4;
// err receives bit 2 if a bounded wait gave up
cudaError_t launch_contract_tc(const ContractArgs<float>& a, bool tf32, int n_sm, float4* coef,
                               unsigned long long* err, int* splits, bool plan_only, int fixed_slices,
                               int skip_copies, cudaStream_t st);
// exclude_degenerate with a tensor-core form: recomputes the b1 = b2 slice partials of the
// Z-triplets with Z2 = Z3 in FP64 (a.partial, a.splits as filled by launch_contract_tc)
cudaError_t launch_contract_diag(const ContractArgs<float>& a, cudaStream_t st);
cudaError_t launch_contract_reduce(const double* partial, int splits, int nz, int nb, int n_max,
                                   double* ups, double* norm, cudaStream_t st);

// ------------------------------------------------------------------ post-processing (FP64)

struct PostArgs {
    int32_t nz, nb, n_max, n_phi, norm_truncate;
    const double* edges;  // device, nb + 1 (arcmin)
    const double* nodes;  // device, nb radial nodes
};

cudaError_t launch_edge_correct(const PostArgs& p, const double* ups, const double* norm,
                                double* gam, unsigned long long* n_singular, cudaStream_t st);
cudaError_t launch_to_gamma(const PostArgs& p, const double* gam, int projection, double* out,
                            cudaStream_t st);
// pixel catalog of the grid-based approximation (Sec. 3.2): per-pixel sums (scratch: 3 n_z npx npy
// doubles) and non-empty flags, then, with rank = exclusive scan of the flags, the compacted pixels
cudaError_t launch_grid_sums(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1, const float* g2,
                             const float* w, const uint8_t* zb, int nz, long long x0, long long y0, long long pq,
                             int npx, int npy, double* scratch, int* flags, int n_sm, cudaStream_t st);
cudaError_t launch_grid_emit(int nz, int npx, int npy, long long x0, long long y0, long long pq, const double* scratch,
                             const int* rank, int32_t* oxq, int32_t* oyq, float* og1, float* og2, float* ow,
                             uint8_t* ozb, int n_sm, cudaStream_t st);
// combined estimator (Sec. 3.3): the pixels that hold a centre galaxy (pmask over the pixel catalog)
cudaError_t launch_grid_combine_map(int64_t nc, const int* centre_idx, const int2* pos, const uint8_t* zs,
                                    long long x0, long long y0, long long pq, int npx, int npy, const int* flags,
                                    const int* rank, int64_t n_pix, uint8_t* pmask, int n_sm, cudaStream_t st);
// rows [b0, b1) of every centre's G, W from the moments of its pixel; also merges the pixel
// catalog's pair counter and error flags into pairs
template <typename T>
cudaError_t launch_grid_gather(int64_t nc, int nz, int nb, int b0, int b1, int n_max, const int* centre_idx,
                               const int2* pos, const uint8_t* zs, long long x0, long long y0, long long pq, int npx,
                               int npy, const int* flags, const int* rank, int64_t nsub, const int* sub_centre_idx,
                               const int* sub_perm, int* inv, int* srow, const cx<T>* Gs, const cx<T>* Ws, cx<T>* G,
                               cx<T>* W, const unsigned long long* sub_pairs, unsigned long long* pairs, int n_sm,
                               cudaStream_t st);
// combined estimator, FFT form of a grid level (csrc/grid_fft.cu): the moments of bins [b0, b1) of
// every centre from the level's pixel sums (gridsum [nz][npy][npx][3], FP64) by FFT convolution
// with the bin kernels; work holds work_bytes of device scratch (grid_fft_work_bytes)
struct FftPlanCache;
FftPlanCache* fft_cache_create();
void fft_cache_destroy(FftPlanCache* c);
size_t grid_fft_work_bytes(int64_t nc, int nz, int nbr, int npx, int npy, double rmax_pixels, size_t elem_bytes,
                           int max_orders, size_t budget);
template <typename T>
cudaError_t grid_fft_moments(FftPlanCache* cache, int64_t nc, int nz, int nb, int b0, int b1, int n_max,
                             const long long* h_e2q, const int* centre_idx, const int2* pos, const uint8_t* zs,
                             long long x0, long long y0, long long pq, int npx, int npy, const double* gridsum,
                             void* work, size_t work_bytes, cx<T>* G, cx<T>* W, int n_sm, cudaStream_t st,
                             const char** what);
// direct estimator of <M_ap^3> (Sec. 5.3): out[centre][radii triple][2] = (numerator, denominator)
cudaError_t launch_map3_direct(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1, const float* g2,
                               const float* w, double quantum, int64_t n_cen, const double* centres, int n_ap,
                               const double* theta, double rcut_factor, double* out, cudaStream_t st);
cudaError_t launch_to_map3(const PostArgs& p, const double* gcen, int n_ap, const double* theta,
                           double* partial, int chunks, double* corr, double* m8,
                           cudaStream_t st);
// the four-equation form: theta3 [3 n_ap][3] and corr3 [n_z^3][3 n_ap][4] complex are scratch,
// partial as for launch_to_map3 with 3 n_ap apertures; m4 [n_z^3][n_ap][4]
cudaError_t launch_to_map3_four(const PostArgs& p, const double* gcen, int n_ap, const double* theta, double* theta3,
                                double* corr3, double* partial, int chunks, double* m4, cudaStream_t st);

// ------------------------------------------------------------------ adjoint of stages (b), (a)

template <typename T>
struct AdjArgs {
    int32_t n_centres, nz, nb, n_max;
    const int32_t* centre_idx;  // sorted position of each centre
    const int2* pos;            // sorted fixed-point positions
    const Pay<T>* pay;          // sorted (w gamma_1, w gamma_2, w)
    const uint8_t* zs;          // sorted zbin (NULL: one bin)
    const int32_t* cell_start;  // as in MomentArgs
    GridDesc g;
    const long long* e2q;
    const cx<T>* G;             // forward moments (order-major)
    const cx<T>* W;
    const double* gups;         // dL/dUpsilon [z3][4][n_max+1][nb][nb] complex
    const double* gnorm;        // dL/dN [z3][2n_max+1][nb][nb] complex
    // the same gradients in the moment precision, group by group (the Upsilon groups in the order
    // of gups, then the N groups): tabY[g][b1][b2] as stored, tabX[g][b2][b1] transposed
    cx<T>* tabX;
    cx<T>* tabY;
    cx<T>* gG;                  // dL/dG, dL/dW (order-major, like G and W)
    cx<T>* gW;
    T* gvw;                     // [n][4] per sorted galaxy: dL/dv (re, im; v = w gamma), direct
                                // dL/dw, unused (16 bytes: one vector atomic per pair in FP32)
    // exclude_degenerate: scratch for the gradients of the j = k sums, [n_z][n_z][nb][4] (NULL:
    // the forward kept the j = k triplets, nothing to do)
    cx<double>* dgs;
};

cudaError_t launch_moments_adjoint_f32(const AdjArgs<float>& a, int64_t n, const int* perm, const float* g1,
                                       const float* g2, const float* w, float* dg1, float* dg2, float* dw,
                                       int n_sm, cudaStream_t st);
cudaError_t launch_moments_adjoint_f64(const AdjArgs<double>& a, int64_t n, const int* perm, const float* g1,
                                       const float* g2, const float* w, float* dg1, float* dg2, float* dw,
                                       int n_sm, cudaStream_t st);

// exclude_degenerate: sums of the j = k triplets per (centre, z, bin) into scratch
// (4 complex values each) and their removal from (ups, norm); AdjArgs carries the catalog state
cudaError_t launch_degenerate_f32(const AdjArgs<float>& a, void* scratch, double* ups, double* norm, int n_sm,
                                  cudaStream_t st);
cudaError_t launch_degenerate_f64(const AdjArgs<double>& a, void* scratch, double* ups, double* norm, int n_sm,
                                  cudaStream_t st);

// adjoints of the FP64 stages (overwrite their outputs)
cudaError_t launch_to_map3_adjoint(const PostArgs& p, int n_ap, const double* theta, const double* gcorr,
                                   const double* gm8, double* ggcen, cudaStream_t st);
cudaError_t launch_to_gamma_adjoint(const PostArgs& p, const double* gphi, int projection, double* ggam,
                                    cudaStream_t st);
cudaError_t launch_edge_correct_adjoint(const PostArgs& p, const double* norm, const double* gam,
                                        const double* ggam, double* scratch, double* gups, double* gnorm,
                                        cudaStream_t st);
size_t edge_correct_adjoint_scratch(const PostArgs& p);

// Kernel attributes and occupancy, set and queried once per (kernel, size) per process: neither
// call is permitted while a stream is being captured into a CUDA graph, so every launch goes
// through these caches (the first, uncaptured, call fills them).
cudaError_t set_smem_attr(const void* func, size_t bytes);
cudaError_t occupancy(int* per_sm, const void* func, int threads, size_t smem);

template <typename F>
inline cudaError_t set_smem_attr(F* func, size_t bytes)
{
    return set_smem_attr(reinterpret_cast<const void*>(func), bytes);
}
template <typename F>
inline cudaError_t occupancy(int* per_sm, F* func, int threads, size_t smem)
{
    return occupancy(per_sm, reinterpret_cast<const void*>(func), threads, smem);
}

__host__ __device__ inline int groups_per_zt(int n_max) { return 4 * (n_max + 1) + 2 * n_max + 1; }

// The moment arrays in device memory are order-major: element (order slot q, centre c, Z z,
// bin b) at ((q * n_centres + c) * nz + z) * nb_pad(nb) + b, the bins padded to an even count so
// that a (q, c, z) row is a multiple of 16 bytes. A group of consecutive orders over a range of
// centres is then a few long contiguous rows (what the tensor-memory-access copies and coalesced
// loads want). Order slots: G q = m + n_max + 3 (m = -n_max-3..n_max-1), W q = m (m = 0..2 n_max).
// The pad bin is never written and never used.
__host__ __device__ inline int nb_pad(int nb) { return (nb + 1) & ~1; }

}  // namespace mp3
