// C ABI of the mp3pcf library and the cell sort (step a0): fixed-point catalog -> galaxies
// ordered by (tomographic bin, cell row, cell column, galaxy index), with cell start offsets.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace mp3 {

static std::mutex g_attr_mu;
static std::map<const void*, size_t> g_smem_set;
static std::map<std::tuple<const void*, int, size_t>, int> g_occ;

cudaError_t set_smem_attr(const void* func, size_t bytes)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_smem_set.find(func);
    if (it != g_smem_set.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_smem_set[func] = bytes;
    return e;
}

cudaError_t occupancy(int* per_sm, const void* func, int threads, size_t smem)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto key = std::make_tuple(func, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, func, threads, smem);
    if (e == cudaSuccess) g_occ[key] = *per_sm;
    return e;
}

// ------------------------------------------------------------------ device buffers

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes < 256 ? 256 : bytes;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename U>
    U* as() const
    {
        return reinterpret_cast<U*>(p);
    }
};

// ------------------------------------------------------------------ a0: cell sort kernels

// fixed-extent mode: every position inside [x0, x1] x [y0, y1] and zbin < nz, else bit 4 of err
__global__ void k_validate(int64_t n, const int32_t* __restrict__ xq, const int32_t* __restrict__ yq,
                           const uint8_t* __restrict__ zb, int nz, long long x0, long long y0, long long x1,
                           long long y1, unsigned long long* err)
{
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const long long x = xq[i], y = yq[i];
        bad |= x < x0 || x > x1 || y < y0 || y > y1 || (zb && zb[i] >= nz);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 4ULL);
}

__global__ void k_or_word(const unsigned long long* __restrict__ src, unsigned long long* dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst |= *src;
}

__global__ void k_bbox_init(int* bb)
{
    bb[0] = INT_MAX;
    bb[1] = INT_MAX;
    bb[2] = INT_MIN;
    bb[3] = INT_MIN;
    bb[4] = 0;  // error flags
}

__global__ void k_bbox(int64_t n, const int32_t* __restrict__ xq, const int32_t* __restrict__ yq,
                       const uint8_t* __restrict__ zb, int nz, int* bb)
{
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = xq[i], y = yq[i];
        mnx = min(mnx, x);
        mny = min(mny, y);
        mxx = max(mxx, x);
        mxy = max(mxy, y);
        if (zb && zb[i] >= nz) bad = 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&bb[0], mnx);
        atomicMin(&bb[1], mny);
        atomicMax(&bb[2], mxx);
        atomicMax(&bb[3], mxy);
        if (bad) atomicOr(&bb[4], 1);
    }
}

// Cell key of every galaxy. With a fixed extent the positions are only validated on the device
// (k_validate raises the error word, reported as EINVAL after the call) and the pipeline runs on;
// a position outside the extent or a z-bin >= nz is therefore clamped to the grid here, so that
// no index derived from it leaves the cell arrays.
__global__ void k_keys(int64_t n, const int32_t* __restrict__ xq, const int32_t* __restrict__ yq,
                       const uint8_t* __restrict__ zb, int nz, GridDesc g, int* __restrict__ key,
                       int* __restrict__ count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const long long dx = max(0LL, (long long)xq[i] - g.x0), dy = max(0LL, (long long)yq[i] - g.y0);
        const int cx_ = (int)min(dx / g.side, (long long)g.ncx - 1);
        const int cy_ = (int)min(dy / g.side, (long long)g.ncy - 1);
        const int z = zb ? min((int)zb[i], nz - 1) : 0;
        const int k = z * g.ncells + cy_ * g.ncx + cx_;
        key[i] = k;
        atomicAdd(&count[k], 1);
    }
}

// exclusive scan in three passes (block scan, scan of block sums, add), deterministic
constexpr int kScanBlock = 1024;

__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int64_t K,
                              int* __restrict__ sums)
{
    __shared__ int wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const int t = threadIdx.x;  // 256 threads x 4 elements
    int v[4];
    int run = 0;
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + t * 4 + q;
        v[q] = i < K ? in[i] : 0;
        run += v[q];
    }
    // warp inclusive scan of per-thread totals
    int x = run;
    const int lane = t & 31, wid = t >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < 8 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < 8) wsum[lane] = s;
    }
    __syncthreads();
    int excl = x - run + (wid > 0 ? wsum[wid - 1] : 0);
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + t * 4 + q;
        if (i < K) out[i] = excl;
        excl += v[q];
    }
    if (t == 255) sums[blockIdx.x] = excl;
}

__global__ void k_scan_sums(int* sums, int nblocks, int* total)
{
    // one block of 1024 threads, sequential over tiles of 1024 sums
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nblocks; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int v = i < nblocks ? sums[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const int incl = x + (wid > 0 ? wsum[wid - 1] : 0);
        if (i < nblocks) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int* __restrict__ out, int64_t K, const int* __restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const int add = sums[blockIdx.x];
    for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
        const int64_t i = base + q;
        if (i < K) out[i] += add;
    }
}

__global__ void k_scatter(int64_t n, const int* __restrict__ key, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ perm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = key[i];
        perm[start[k] + atomicAdd(&fill[k], 1)] = (int)i;
    }
}

// atomics leave the order inside a cell arbitrary; restore increasing galaxy index so that the
// whole pipeline is deterministic
__global__ void k_cell_order(int64_t K, const int* __restrict__ start, int* __restrict__ perm)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < K;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int a = start[c], b = start[c + 1];
        for (int i = a + 1; i < b; ++i) {
            const int v = perm[i];
            int j = i - 1;
            while (j >= a && perm[j] > v) {
                perm[j + 1] = perm[j];
                --j;
            }
            perm[j + 1] = v;
        }
    }
}

template <typename T>
__global__ void k_gather(int64_t n, const int* __restrict__ perm, const int32_t* __restrict__ xq,
                         const int32_t* __restrict__ yq, const float* __restrict__ g1,
                         const float* __restrict__ g2, const float* __restrict__ w,
                         const uint8_t* __restrict__ zb, const uint8_t* __restrict__ mask,
                         int2* __restrict__ pos, Pay<T>* __restrict__ pay,
                         uint8_t* __restrict__ zs, int* __restrict__ cflag, int nz)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n;
         d += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[d];
        pos[d] = make_int2(xq[i], yq[i]);
        const T wi = (T)w[i];
        pay[d] = Pay<T>{wi * (T)g1[i], wi * (T)g2[i], wi, T(0)};
        zs[d] = zb ? (uint8_t)min((int)zb[i], nz - 1) : 0;  // clamped like the cell key (k_keys)
        cflag[d] = mask ? (mask[i] != 0) : 1;
    }
}

__global__ void k_mask_flags(int64_t n, const uint8_t* __restrict__ mask, int* __restrict__ f)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = mask ? (mask[i] != 0) : 1;
}

// first centre of each z-bin in the centre list (sorted by z-bin first): the sorted index of the
// first galaxy of z-bin z is cell_start[z * ncells], its rank among the centres crank[] of it
__global__ void k_zrange(int nz, int64_t ncells, const int* __restrict__ cell_start, const int* __restrict__ crank,
                         int* __restrict__ zrange)
{
    for (int z = threadIdx.x; z <= nz; z += blockDim.x) zrange[z] = crank[cell_start[(int64_t)z * ncells]];
}

// centre list in sorted order and, for each centre, its row in galaxy-index order
__global__ void k_centres(int64_t n, const int* __restrict__ perm, const int* __restrict__ cflag,
                          const int* __restrict__ crank, const int* __restrict__ orank,
                          int* __restrict__ centre_idx, int* __restrict__ crow)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n;
         d += (int64_t)gridDim.x * blockDim.x) {
        if (cflag[d]) {
            const int r = crank[d];
            centre_idx[r] = (int)d;
            crow[r] = orank[perm[d]];
        }
    }
}

template <typename T>
__global__ void k_copy_rows(int64_t nc, int nz, int nb, int len, const int* __restrict__ crow,
                            const cx<T>* __restrict__ src, cx<T>* __restrict__ dst)
{
    // order-major src[q][c][z][nb_pad] (centres in sorted order) -> dst[crow[c]][z][b][q]
    const int nbp = nb_pad(nb);
    const int64_t total = (int64_t)len * nc * nz * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % nb);
        int64_t r = t / nb;
        const int z = (int)(r % nz);
        r /= nz;
        const int64_t c = r % nc;
        const int q = (int)(r / nc);
        dst[(((int64_t)crow[c] * nz + z) * nb + b) * len + q] = src[(((int64_t)q * nc + c) * nz + z) * nbp + b];
    }
}

}  // namespace mp3

using namespace mp3;

// ------------------------------------------------------------------ context

struct mp3pcf_ctx {
    mp3pcf_config cfg;
    cudaStream_t st = nullptr;
    int device = 0;
    int n_sm = 0;
    bool fp64 = false;
    std::vector<double> edges, nodes;
    std::vector<long long> e2q;
    std::string err;
    // catalog state of the last accumulate call
    int64_t n = 0;
    int64_t n_centres = 0;
    GridDesc grid{};
    // fixed patch extent (fixed-point x0, y0, x1, y1): no host round trip for the cell grid
    bool fixed_extent = false;
    int64_t ext[4] = {0, 0, 0, 0};
    DevBuf bups, bnorm, bgam, bgcen, berr;  // batch workspace
    int64_t graph_launches = 0, graph_instantiations = 0;
    cudaStream_t batch_st = nullptr;  // capturable stream of mp3pcf_run_batch (created on first use)
    // fault injection on the host side (tests of failure detection): see mp3pcf_inject
    bool inject_wait_timeout = false, inject_alloc_failure = false;
    cudaEvent_t batch_ev[2] = {nullptr, nullptr};
    DevBuf d_e2q, d_edges, d_nodes;
    DevBuf bb, key, count, fill, scan_sums, scan_total, perm, pos, pay, zs;
    DevBuf cflag, crank, oflag, orank, centre_idx, crow;
    DevBuf G, W, pairs, partial, singular, m3partial, m3four, ccoef;
    DevBuf gG, gW, gv, gtab, adjscratch;  // adjoint workspace
    DevBuf degen;                       // exclude_degenerate sums per (centre, z, bin)
    DevBuf degen_grad;                  // their gradient sums per (Z1, z, bin) in the adjoint
    DevBuf zrange;                      // [nz + 1] centre range of each z-bin
    DevBuf fftwork;                     // FFT grid moments: padded fields, kernels, products
    FftPlanCache* fft = nullptr;        // cuFFT plans of the FFT grid moments
    DevBuf gridsum;                     // per-pixel FP64 sums of the grid-based approximation
    DevBuf gridflag;                    // its non-empty flags and their exclusive scan
    // combined estimator: the moments of the last accumulate call mix discrete and grid bins
    bool combined = false;
    long long bbox[4] = {0, 0, 0, 0};   // extent (x0, y0, x1, y1) of the last accumulate call
    mp3pcf_ctx* sub = nullptr;          // context of the pixel catalogs (created on first use)
    DevBuf pix, pixinv;                 // a pixel catalog (SoA); its catalog index -> moment row, then each centre's row
    // tracing: per-stage event pairs and kernel-launch counts
    bool timing = false;
    int64_t launches[6] = {0, 0, 0, 0, 0, 0};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    std::vector<cudaEvent_t> pool;
};

enum { ST_SORT = 0, ST_MOMENTS = 1, ST_CONTRACT = 2, ST_EDGE = 3, ST_GAMMA = 4, ST_MAP3 = 5 };

static cudaEvent_t stage_begin(mp3pcf_ctx* ctx)
{
    if (!ctx->timing) return nullptr;
    cudaEvent_t e = nullptr;
    if (!ctx->pool.empty()) {
        e = ctx->pool.back();
        ctx->pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, ctx->st);
    return e;
}

static void stage_end(mp3pcf_ctx* ctx, int stage, cudaEvent_t b)
{
    if (!b) return;
    cudaEvent_t e = stage_begin(ctx);
    if (!e) {
        ctx->pool.push_back(b);
        return;
    }
    ctx->ev.push_back({stage, {b, e}});
}

// records the end event of a stage when it goes out of scope
// NVTX ranges (visible to nsys / ncu range filters; free without a tool): one per stage call and
// one around each public entry point that spans stages
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static const char* const kStageNames[6] = {"mp3pcf sort", "mp3pcf moments", "mp3pcf contract",
                                           "mp3pcf edge_correct", "mp3pcf to_gamma", "mp3pcf to_map3"};

struct StageScope {
    mp3pcf_ctx* ctx;
    int stage;
    cudaEvent_t b;
    StageScope(mp3pcf_ctx* c, int s) : ctx(c), stage(s), b(stage_begin(c)) { nvtxRangePushA(kStageNames[s]); }
    ~StageScope()
    {
        stage_end(ctx, stage, b);
        nvtxRangePop();
    }
};

static mp3pcf_status fail(mp3pcf_ctx* c, mp3pcf_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

#define MP3_CK(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MP3PCF_ENOMEM : MP3PCF_ECUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

static bool config_valid(const mp3pcf_config* c, std::string* why)
{
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (!c) return bad("null config");
    if (c->n_bins < 1 || c->n_bins > kMaxBins) return bad("n_bins out of range");
    if (!(c->theta_min > 0) || !(c->theta_max > c->theta_min) || !std::isfinite(c->theta_max))
        return bad("need 0 < theta_min < theta_max");
    if (c->n_max < 0 || c->n_max > kMaxNmax) return bad("n_max out of range");
    if (c->n_phi < 1 || c->n_phi > 100000) return bad("n_phi out of range");
    if (c->n_z < 1 || c->n_z > kMaxNz) return bad("n_z out of range");
    if (!(c->quantum > 0) || !std::isfinite(c->quantum)) return bad("quantum must be > 0");
    if (c->precision < MP3PCF_FP64 || c->precision > MP3PCF_FP32_TF32X3) return bad("precision");
    if (c->norm_truncate != 0 && c->norm_truncate != 1) return bad("norm_truncate");
    if (c->radial_nodes != 0 && c->radial_nodes != 1) return bad("radial_nodes");
    if (c->cell_occupancy < 0 || c->cell_occupancy > 64) return bad("cell_occupancy out of range");
    if (c->contract_slices < 0 || c->contract_slices > 64) return bad("contract_slices out of range");
    if (c->exclude_degenerate != 0 && c->exclude_degenerate != 1) return bad("exclude_degenerate");
    if (c->grid_fft != 0 && c->grid_fft != 1) return bad("grid_fft");
    if (c->reserved != 0) return bad("reserved fields must be zero");
    const double t = c->theta_max / c->quantum;
    if (t * t >= 9.0e18) return bad("theta_max / quantum too large");
    return true;
}

// bin edges and their exact squared fixed-point values (same definition the header states)
static void host_edges(const mp3pcf_config* c, std::vector<double>& e, std::vector<long long>& e2)
{
    e.resize(c->n_bins + 1);
    e2.resize(c->n_bins + 1);
    for (int b = 0; b <= c->n_bins; ++b) {
        const double eb = c->theta_min * pow(c->theta_max / c->theta_min, (double)b / c->n_bins);
        const double t = eb / c->quantum;
        e[b] = eb;
        e2[b] = (long long)ceil(t * t);
    }
}

template <typename T>
static mp3pcf_status degenerate_t(mp3pcf_ctx* ctx, double* ups, double* norm);

extern "C" {

mp3pcf_status mp3pcf_bin_edges(const mp3pcf_config* cfg, double* h_edges, int64_t* h_edges2_q)
{
    if (!config_valid(cfg, nullptr)) return MP3PCF_EINVAL;
    std::vector<double> e;
    std::vector<long long> e2;
    host_edges(cfg, e, e2);
    for (int b = 0; b <= cfg->n_bins; ++b) {
        if (h_edges) h_edges[b] = e[b];
        if (h_edges2_q) h_edges2_q[b] = (int64_t)e2[b];
    }
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_create(const mp3pcf_config* cfg, void* stream, mp3pcf_ctx** out)
{
    if (!out) return MP3PCF_EINVAL;
    *out = nullptr;
    std::string why;
    if (!config_valid(cfg, &why)) return MP3PCF_EINVAL;
    mp3pcf_ctx* ctx = new mp3pcf_ctx();
    ctx->cfg = *cfg;
    ctx->st = (cudaStream_t)stream;
    ctx->fp64 = cfg->precision == MP3PCF_FP64;
    host_edges(cfg, ctx->edges, ctx->e2q);
    ctx->nodes.resize(cfg->n_bins);
    for (int b = 0; b < cfg->n_bins; ++b)
        ctx->nodes[b] = cfg->radial_nodes ? sqrt(ctx->edges[b] * ctx->edges[b + 1])
                                          : 0.5 * (ctx->edges[b] + ctx->edges[b + 1]);
    auto cleanup = [&](mp3pcf_status s) {
        mp3pcf_destroy(ctx);
        return s;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return cleanup(MP3PCF_ECUDA);
    if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return cleanup(MP3PCF_ECUDA);
    const int nb = cfg->n_bins;
    if (ctx->d_e2q.ensure(sizeof(long long) * (nb + 1)) != cudaSuccess ||
        ctx->d_edges.ensure(sizeof(double) * (nb + 1)) != cudaSuccess ||
        ctx->d_nodes.ensure(sizeof(double) * nb) != cudaSuccess ||
        ctx->bb.ensure(sizeof(int) * 8) != cudaSuccess || ctx->pairs.ensure(24) != cudaSuccess ||
        ctx->singular.ensure(8) != cudaSuccess)
        return cleanup(MP3PCF_ENOMEM);
    if (cudaMemcpy(ctx->d_e2q.p, ctx->e2q.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_edges.p, ctx->edges.data(), sizeof(double) * (nb + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_nodes.p, ctx->nodes.data(), sizeof(double) * nb, cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(MP3PCF_ECUDA);
    *out = ctx;
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_destroy(mp3pcf_ctx* ctx)
{
    if (!ctx) return MP3PCF_OK;
    cudaStreamSynchronize(ctx->st);
    DevBuf* bufs[] = {&ctx->d_e2q, &ctx->d_edges, &ctx->d_nodes, &ctx->bb, &ctx->key,
                      &ctx->count, &ctx->fill, &ctx->scan_sums, &ctx->scan_total, &ctx->perm,
                      &ctx->pos, &ctx->pay, &ctx->zs, &ctx->cflag,
                      &ctx->crank, &ctx->oflag, &ctx->orank, &ctx->centre_idx, &ctx->crow,
                      &ctx->G, &ctx->W, &ctx->pairs, &ctx->partial, &ctx->singular,
                      &ctx->m3partial, &ctx->m3four, &ctx->fftwork, &ctx->ccoef, &ctx->gG, &ctx->gW, &ctx->gv, &ctx->gtab,
                      &ctx->adjscratch, &ctx->degen, &ctx->degen_grad, &ctx->zrange, &ctx->gridsum, &ctx->gridflag, &ctx->bups, &ctx->bnorm,
                      &ctx->bgam, &ctx->bgcen, &ctx->berr, &ctx->pix, &ctx->pixinv};
    for (DevBuf* b : bufs) b->release();
    if (ctx->fft) fft_cache_destroy(ctx->fft);
    if (ctx->sub) mp3pcf_destroy(ctx->sub);
    if (ctx->batch_st) cudaStreamDestroy(ctx->batch_st);
    for (cudaEvent_t ev : ctx->batch_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& pr : ctx->ev) {
        cudaEventDestroy(pr.second.first);
        cudaEventDestroy(pr.second.second);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    delete ctx;
    return MP3PCF_OK;
}

const char* mp3pcf_last_error(const mp3pcf_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

}  // extern "C"

// exclusive scan of K ints from `in` to `out` (out has K+1 entries; out[K] = total)
static mp3pcf_status scan_exclusive(mp3pcf_ctx* ctx, const int* in, int* out, int64_t K)
{
    const int64_t nblk = (K + kScanBlock - 1) / kScanBlock;
    ctx->launches[ST_SORT] += nblk > 0 ? 3 : 1;
    MP3_CK(ctx->scan_sums.ensure(sizeof(int) * (nblk + 1)));
    if (nblk > 0) {
        k_scan_blocks<<<(unsigned)nblk, 256, 0, ctx->st>>>(in, out, K, ctx->scan_sums.as<int>());
        MP3_CK(cudaGetLastError());
    }
    k_scan_sums<<<1, 1024, 0, ctx->st>>>(ctx->scan_sums.as<int>(), (int)nblk, out + K);
    MP3_CK(cudaGetLastError());
    if (nblk > 0) {
        k_scan_add<<<(unsigned)nblk, 256, 0, ctx->st>>>(out, K, ctx->scan_sums.as<int>());
        MP3_CK(cudaGetLastError());
    }
    return MP3PCF_OK;
}

static unsigned grid1d(int64_t n, int n_sm)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)n_sm * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename T>
static mp3pcf_status accumulate_t(mp3pcf_ctx* ctx, int64_t n, const int32_t* xq, const int32_t* yq,
                                  const float* g1, const float* g2, const float* w,
                                  const uint8_t* zb, const uint8_t* mask, int b_lo, int b_hi)
{
    const mp3pcf_config& c = ctx->cfg;
    const int nz = c.n_z, nb = c.n_bins;
    cudaStream_t st = ctx->st;
    ctx->n = n;
    ctx->n_centres = 0;
    ctx->combined = false;
    MP3_CK(cudaMemsetAsync(ctx->pairs.p, 0, 24, st));
    if (n == 0) return MP3PCF_OK;
    if (ctx->inject_alloc_failure) return fail(ctx, MP3PCF_ENOMEM, "injected allocation failure");

    // ---- extent of the catalog: given (fixed-extent mode, validated on the device), or one
    // host round trip
    NvtxRange nvtx_acc("mp3pcf accumulate_moments");
    cudaEvent_t t_sort = stage_begin(ctx);
    long long bb[5];
    if (ctx->fixed_extent) {
        for (int i = 0; i < 4; ++i) bb[i] = ctx->ext[i];
        bb[4] = 0;
        ctx->launches[ST_SORT] += 1;
        k_validate<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, xq, yq, zb, nz, bb[0], bb[1], bb[2], bb[3],
                                                          ctx->pairs.as<unsigned long long>() + 1);
        MP3_CK(cudaGetLastError());
    } else {
        ctx->launches[ST_SORT] += 2;
        k_bbox_init<<<1, 1, 0, st>>>(ctx->bb.as<int>());
        k_bbox<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, xq, yq, zb, nz, ctx->bb.as<int>());
        MP3_CK(cudaGetLastError());
        int hb[5];
        MP3_CK(cudaMemcpyAsync(hb, ctx->bb.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
        MP3_CK(cudaStreamSynchronize(st));
        for (int i = 0; i < 5; ++i) bb[i] = hb[i];
    }
    if (bb[4]) {
        stage_end(ctx, ST_SORT, t_sort);
        return fail(ctx, MP3PCF_EINVAL, "zbin value >= n_z");
    }
    for (int i = 0; i < 4; ++i) ctx->bbox[i] = bb[i];
    const long long ex = (long long)bb[2] - bb[0], ey = (long long)bb[3] - bb[1];
    if (ex >= (1LL << 24) || ey >= (1LL << 24)) {
        stage_end(ctx, ST_SORT, t_sort);
        return fail(ctx, MP3PCF_EINVAL, "patch extent must be below 2^24 position quanta");
    }

    // ---- cell grid: ~4 galaxies per cell and bin, and at most kMaxRows rows per annulus of the
    // computed bins
    const double R = sqrt((double)ctx->e2q[b_hi]);
    const double area = (double)(ex + 1) * (double)(ey + 1);
    const double occ = c.cell_occupancy > 0 ? (double)c.cell_occupancy : 4.0;
    double side = sqrt(area * occ / std::max(1.0, (double)n / nz));
    side = std::max(side, (2.0 * R + 16.0) / (kMaxRows - 4));
    side = std::max(side, sqrt(area * nz / (double)(1 << 26)));
    side = std::max(side, 1.0);
    GridDesc g;
    g.x0 = bb[0];
    g.y0 = bb[1];
    g.side = (int32_t)ceil(side);
    g.ncx = (int32_t)(ex / g.side + 1);
    g.ncy = (int32_t)(ey / g.side + 1);
    g.ncells = g.ncx * g.ncy;
    ctx->grid = g;
    const int64_t K = (int64_t)nz * g.ncells;

    // ---- counting sort by (zbin, cell)
    MP3_CK(ctx->key.ensure(sizeof(int) * n));
    MP3_CK(ctx->count.ensure(sizeof(int) * (K + 1)));
    MP3_CK(ctx->fill.ensure(sizeof(int) * (K + 1)));
    MP3_CK(ctx->perm.ensure(sizeof(int) * n));
    MP3_CK(ctx->pos.ensure(sizeof(int2) * n));
    MP3_CK(ctx->pay.ensure(sizeof(Pay<T>) * n));
    MP3_CK(ctx->zs.ensure(n));
    MP3_CK(ctx->cflag.ensure(sizeof(int) * (n + 1)));
    MP3_CK(ctx->crank.ensure(sizeof(int) * (n + 1)));
    MP3_CK(ctx->oflag.ensure(sizeof(int) * (n + 1)));
    MP3_CK(ctx->orank.ensure(sizeof(int) * (n + 1)));
    MP3_CK(ctx->centre_idx.ensure(sizeof(int) * n));
    MP3_CK(ctx->crow.ensure(sizeof(int) * n));
    MP3_CK(cudaMemsetAsync(ctx->fill.p, 0, sizeof(int) * (K + 1), st));
    ctx->launches[ST_SORT] += 6;
    k_keys<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, xq, yq, zb, nz, g, ctx->key.as<int>(), ctx->fill.as<int>());
    MP3_CK(cudaGetLastError());
    if (mp3pcf_status s = scan_exclusive(ctx, ctx->fill.as<int>(), ctx->count.as<int>(), K)) return s;
    MP3_CK(cudaMemsetAsync(ctx->fill.p, 0, sizeof(int) * (K + 1), st));
    k_scatter<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, ctx->key.as<int>(), ctx->count.as<int>(),
                                                    ctx->fill.as<int>(), ctx->perm.as<int>());
    k_cell_order<<<grid1d(K, ctx->n_sm), 256, 0, st>>>(K, ctx->count.as<int>(), ctx->perm.as<int>());
    k_gather<T><<<grid1d(n, ctx->n_sm), 256, 0, st>>>(
        n, ctx->perm.as<int>(), xq, yq, g1, g2, w, zb, mask, ctx->pos.as<int2>(), ctx->pay.as<Pay<T>>(),
        ctx->zs.as<uint8_t>(), ctx->cflag.as<int>(), nz);
    MP3_CK(cudaGetLastError());

    // ---- centre list (sorted order) and each centre's row in galaxy-index order
    if (mp3pcf_status s = scan_exclusive(ctx, ctx->cflag.as<int>(), ctx->crank.as<int>(), n)) return s;
    k_mask_flags<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, mask, ctx->oflag.as<int>());
    if (mp3pcf_status s = scan_exclusive(ctx, ctx->oflag.as<int>(), ctx->orank.as<int>(), n)) return s;
    k_centres<<<grid1d(n, ctx->n_sm), 256, 0, st>>>(n, ctx->perm.as<int>(), ctx->cflag.as<int>(),
                                                    ctx->crank.as<int>(), ctx->orank.as<int>(),
                                                    ctx->centre_idx.as<int>(), ctx->crow.as<int>());
    MP3_CK(cudaGetLastError());
    if (nz > 1) {
        MP3_CK(ctx->zrange.ensure(sizeof(int) * (nz + 1)));
        k_zrange<<<1, 32, 0, st>>>(nz, g.ncells, ctx->count.as<int>(), ctx->crank.as<int>(), ctx->zrange.as<int>());
        MP3_CK(cudaGetLastError());
        ctx->launches[ST_SORT] += 1;
    }
    int nc = (int)n;
    if (mask) {
        MP3_CK(cudaMemcpyAsync(&nc, ctx->crank.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        MP3_CK(cudaStreamSynchronize(st));
    }
    ctx->n_centres = nc;
    stage_end(ctx, ST_SORT, t_sort);
    if (nc == 0) return MP3PCF_OK;

    // ---- stage (a)
    MP3_CK(ctx->G.ensure(sizeof(cx<T>) * (size_t)(2 * c.n_max + 3) * nc * nz * nb_pad(nb)));
    MP3_CK(ctx->W.ensure(sizeof(cx<T>) * (size_t)(2 * c.n_max + 1) * nc * nz * nb_pad(nb)));
    MomentArgs<T> a;
    a.n_centres = nc;
    a.centre_idx = ctx->centre_idx.as<int>();
    a.pos = ctx->pos.as<int2>();
    a.pay = ctx->pay.as<Pay<T>>();
    a.cell_start = ctx->count.as<int>();
    a.g = g;
    a.nz = nz;
    a.nb = b_hi - b_lo;
    a.nbp = nb_pad(nb);
    a.n_max = c.n_max;
    a.e2q = ctx->d_e2q.as<long long>() + b_lo;
    a.G = ctx->G.as<cx<T>>() + b_lo;
    a.W = ctx->W.as<cx<T>>() + b_lo;
    a.pairs = ctx->pairs.as<unsigned long long>();
    a.queue = ctx->pairs.as<unsigned long long>() + 2;
    if (b_lo >= b_hi) return MP3PCF_OK;
    cudaError_t e;
    {
        StageScope sc(ctx, ST_MOMENTS);
        ctx->launches[ST_MOMENTS] += 1;
        if constexpr (sizeof(T) == 8)
            e = launch_moments_f64(a, ctx->n_sm, st);
        else
            e = launch_moments_f32(a, ctx->n_sm, st);
    }
    MP3_CK(e);
    return MP3PCF_OK;
}

extern "C" {

mp3pcf_status mp3pcf_accumulate_moments(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq,
                                        const int32_t* d_yq, const float* d_g1, const float* d_g2,
                                        const float* d_w, const uint8_t* d_zbin,
                                        const uint8_t* d_centre_mask)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->err.clear();
    if (n < 0 || n > INT_MAX / 2) return fail(ctx, MP3PCF_EINVAL, "n out of range");
    if (n > 0 && (!d_xq || !d_yq || !d_g1 || !d_g2 || !d_w))
        return fail(ctx, MP3PCF_EINVAL, "null catalog pointer");
    if (ctx->cfg.n_z > 1 && n > 0 && !d_zbin)
        return fail(ctx, MP3PCF_EINVAL, "n_z > 1 needs zbin");
    const int nb = ctx->cfg.n_bins;
    if (ctx->fp64) return accumulate_t<double>(ctx, n, d_xq, d_yq, d_g1, d_g2, d_w, d_zbin, d_centre_mask, 0, nb);
    return accumulate_t<float>(ctx, n, d_xq, d_yq, d_g1, d_g2, d_w, d_zbin, d_centre_mask, 0, nb);
}

}  // extern "C"

// combined estimator (Sec. 3.3): bins [0, b_start[0]) from the galaxies, bins [b_start[l],
// b_start[l + 1]) (the last level to n_bins) from the pixel catalog of side pixel_q[l] at the
// pixel of each centre galaxy; the pixel catalogs' moments run in a second context
template <typename T>
static mp3pcf_status combined_t(mp3pcf_ctx* ctx, int64_t n, const int32_t* xq, const int32_t* yq, const float* g1,
                                const float* g2, const float* w, const uint8_t* zb, const uint8_t* mask, int L,
                                const int32_t* b_start, const int64_t* pixel_q)
{
    const mp3pcf_config& c = ctx->cfg;
    const int nz = c.n_z, nb = c.n_bins;
    if (mp3pcf_status s = accumulate_t<T>(ctx, n, xq, yq, g1, g2, w, zb, mask, 0, b_start[0])) return s;
    const int64_t nc = ctx->n_centres;
    if (nc == 0) {
        ctx->combined = true;
        return MP3PCF_OK;
    }
    if (!ctx->sub) {
        if (mp3pcf_status s = mp3pcf_create(&ctx->cfg, ctx->st, &ctx->sub))
            return fail(ctx, s, "could not create the pixel catalogs' context");
    }
    mp3pcf_ctx* sub = ctx->sub;
    const long long x0 = ctx->bbox[0], y0 = ctx->bbox[1];
    for (int l = 0; l < L; ++l) {
        const long long pq = pixel_q[l];
        const int b0 = b_start[l], b1 = l + 1 < L ? b_start[l + 1] : nb;
        const long long npx = (ctx->bbox[2] - x0) / pq + 1, npy = (ctx->bbox[3] - y0) / pq + 1;
        const long long npix = (long long)nz * npx * npy;
        if (npix > 0x7fffffffLL) return fail(ctx, MP3PCF_EINVAL, "a grid level has more than 2^31 - 1 pixels");
        if (x0 + npx * pq > INT_MAX || y0 + npy * pq > INT_MAX)
            return fail(ctx, MP3PCF_EINVAL, "a grid level lies outside the fixed-point range");
        // pixel catalog (SoA xq, yq, g1, g2, w, zbin, centre mask) and the galaxies' pixels
        MP3_CK(ctx->gridsum.ensure(sizeof(double) * 3 * (size_t)npix));
        MP3_CK(ctx->gridflag.ensure(sizeof(int) * 2 * ((size_t)npix + 1)));
        MP3_CK(ctx->pix.ensure(22 * (size_t)npix));
        MP3_CK(ctx->pixinv.ensure(sizeof(int) * ((size_t)npix + (size_t)nc)));
        int* flags = ctx->gridflag.as<int>();
        int* rank = flags + npix + 1;
        char* pb = ctx->pix.as<char>();
        int32_t* pxq = (int32_t*)pb;
        int32_t* pyq = (int32_t*)(pb + 4 * npix);
        float* pg1 = (float*)(pb + 8 * npix);
        float* pg2 = (float*)(pb + 12 * npix);
        float* pw = (float*)(pb + 16 * npix);
        uint8_t* pzb = (uint8_t*)(pb + 20 * npix);
        uint8_t* pmask = (uint8_t*)(pb + 21 * npix);
        const uint8_t* czs = nz > 1 ? ctx->zs.as<uint8_t>() : nullptr;
        ctx->launches[ST_MOMENTS] += 8;
        MP3_CK(launch_grid_sums(n, xq, yq, g1, g2, w, zb, nz, x0, y0, pq, (int)npx, (int)npy,
                                ctx->gridsum.as<double>(), flags, ctx->n_sm, ctx->st));
        if (c.grid_fft) {
            // the level's moments by FFT convolution of the gridded fields (no pixel catalog)
            if (!ctx->fft) ctx->fft = fft_cache_create();
            std::vector<long long> e2q(nb + 1);
            if (mp3pcf_bin_edges(&c, nullptr, reinterpret_cast<int64_t*>(e2q.data())) != MP3PCF_OK)
                return fail(ctx, MP3PCF_EINVAL, "bin edges");
            const size_t wb = grid_fft_work_bytes(nc, nz, b1 - b0, (int)npx, (int)npy,
                                                  std::sqrt((double)e2q[b1]) / (double)pq, sizeof(T),
                                                  std::max(2 * c.n_max, c.n_max + 3) + 1, (size_t)6 << 30);
            MP3_CK(ctx->fftwork.ensure(wb));
            ctx->launches[ST_MOMENTS] += 2;
            const char* what = "";
            const cudaError_t fe = grid_fft_moments<T>(
                ctx->fft, nc, nz, nb, b0, b1, c.n_max, e2q.data(), ctx->centre_idx.as<int>(), ctx->pos.as<int2>(), czs,
                x0, y0, pq, (int)npx, (int)npy, ctx->gridsum.as<double>(), ctx->fftwork.p, wb, ctx->G.as<cx<T>>(),
                ctx->W.as<cx<T>>(), ctx->n_sm, ctx->st, &what);
            if (fe != cudaSuccess) return fail(ctx, MP3PCF_ECUDA, (std::string("FFT grid moments: ") + what).c_str());
            continue;
        }
        if (mp3pcf_status s = scan_exclusive(ctx, flags, rank, npix)) return s;
        MP3_CK(launch_grid_emit(nz, (int)npx, (int)npy, x0, y0, pq, ctx->gridsum.as<double>(), rank, pxq, pyq, pg1,
                                pg2, pw, nz > 1 ? pzb : nullptr, ctx->n_sm, ctx->st));
        MP3_CK(launch_grid_combine_map(nc, ctx->centre_idx.as<int>(), ctx->pos.as<int2>(), czs, x0, y0, pq, (int)npx,
                                       (int)npy, flags, rank, npix, pmask, ctx->n_sm, ctx->st));
        int cnt = 0;
        MP3_CK(cudaMemcpyAsync(&cnt, rank + npix, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        MP3_CK(cudaStreamSynchronize(ctx->st));
        if (cnt > INT_MAX / 2) return fail(ctx, MP3PCF_EINVAL, "a grid level has more than 2^30 non-empty pixels");
        // the pixel catalog's moments of this level's bins
        int64_t before[6];
        for (int i = 0; i < 6; ++i) before[i] = sub->launches[i];
        sub->inject_wait_timeout = ctx->inject_wait_timeout;
        if (mp3pcf_status s = accumulate_t<T>(sub, cnt, pxq, pyq, pg1, pg2, pw, nz > 1 ? pzb : nullptr, pmask, b0, b1))
            return fail(ctx, s, ("pixel catalog: " + sub->err).c_str());
        for (int i = 0; i < 6; ++i) ctx->launches[i] += sub->launches[i] - before[i];
        ctx->launches[ST_MOMENTS] += 4;
        MP3_CK(launch_grid_gather<T>(nc, nz, nb, b0, b1, c.n_max, ctx->centre_idx.as<int>(), ctx->pos.as<int2>(), czs,
                                     x0, y0, pq, (int)npx, (int)npy, flags, rank, sub->n_centres,
                                     sub->centre_idx.as<int>(), sub->perm.as<int>(), ctx->pixinv.as<int>(),
                                     ctx->pixinv.as<int>() + npix, sub->G.as<cx<T>>(), sub->W.as<cx<T>>(), ctx->G.as<cx<T>>(), ctx->W.as<cx<T>>(),
                                     sub->pairs.as<unsigned long long>(), ctx->pairs.as<unsigned long long>(),
                                     ctx->n_sm, ctx->st));
    }
    ctx->combined = true;
    return MP3PCF_OK;
}

extern "C" {

mp3pcf_status mp3pcf_accumulate_moments_combined(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq,
                                                 const int32_t* d_yq, const float* d_g1, const float* d_g2,
                                                 const float* d_w, const uint8_t* d_zbin,
                                                 const uint8_t* d_centre_mask, int32_t n_levels,
                                                 const int32_t* h_b_start, const int64_t* h_pixel_q)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->err.clear();
    const int nb = ctx->cfg.n_bins;
    if (n < 0 || n > INT_MAX / 2) return fail(ctx, MP3PCF_EINVAL, "n out of range");
    if (n > 0 && (!d_xq || !d_yq || !d_g1 || !d_g2 || !d_w))
        return fail(ctx, MP3PCF_EINVAL, "null catalog pointer");
    if (ctx->cfg.n_z > 1 && n > 0 && !d_zbin)
        return fail(ctx, MP3PCF_EINVAL, "n_z > 1 needs zbin");
    if (n_levels < 1 || !h_b_start || !h_pixel_q) return fail(ctx, MP3PCF_EINVAL, "no grid level");
    for (int l = 0; l < n_levels; ++l) {
        if (h_pixel_q[l] < 1 || h_pixel_q[l] > INT_MAX) return fail(ctx, MP3PCF_EINVAL, "pixel_q out of range");
        if (h_b_start[l] < 0 || h_b_start[l] >= nb || (l > 0 && h_b_start[l] <= h_b_start[l - 1]))
            return fail(ctx, MP3PCF_EINVAL, "b_start must increase strictly within [0, n_bins)");
    }
    if (ctx->cfg.exclude_degenerate)
        return fail(ctx, MP3PCF_EUNSUPPORTED, "the combined estimator does not take exclude_degenerate");
    NvtxRange nvtx("mp3pcf accumulate_moments_combined");
    if (ctx->fp64)
        return combined_t<double>(ctx, n, d_xq, d_yq, d_g1, d_g2, d_w, d_zbin, d_centre_mask, n_levels, h_b_start,
                                  h_pixel_q);
    return combined_t<float>(ctx, n, d_xq, d_yq, d_g1, d_g2, d_w, d_zbin, d_centre_mask, n_levels, h_b_start,
                             h_pixel_q);
}

mp3pcf_status mp3pcf_counts(mp3pcf_ctx* ctx, int64_t* h_n_centres, int64_t* h_n_pairs)
{
    if (!ctx) return MP3PCF_EINVAL;
    if (h_n_centres) *h_n_centres = ctx->n_centres;
    unsigned long long p[2] = {0, 0};
    MP3_CK(cudaMemcpyAsync(p, ctx->pairs.p, 16, cudaMemcpyDeviceToHost, ctx->st));
    MP3_CK(cudaStreamSynchronize(ctx->st));
    if (h_n_pairs) *h_n_pairs = (int64_t)p[0];
    if (p[1] & 4ULL) return fail(ctx, MP3PCF_EINVAL, "a galaxy lies outside the fixed extent or has zbin >= n_z");
    if (p[1]) return fail(ctx, MP3PCF_ETIMEOUT, "a bounded device wait in the moment or contraction kernel gave up");
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_copy_moments(mp3pcf_ctx* ctx, void* d_G, void* d_W)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->err.clear();
    const int64_t nc = ctx->n_centres;
    if (nc == 0) return MP3PCF_OK;
    const mp3pcf_config& c = ctx->cfg;
    const int nz = c.n_z, nb = c.n_bins, lg = 2 * c.n_max + 3, lw = 2 * c.n_max + 1;
    const unsigned gr = grid1d(nc * nz * nb * lg, ctx->n_sm);
    if (ctx->fp64) {
        if (d_G) k_copy_rows<double><<<gr, 256, 0, ctx->st>>>(nc, nz, nb, lg, ctx->crow.as<int>(), ctx->G.as<cx<double>>(), (cx<double>*)d_G);
        if (d_W) k_copy_rows<double><<<gr, 256, 0, ctx->st>>>(nc, nz, nb, lw, ctx->crow.as<int>(), ctx->W.as<cx<double>>(), (cx<double>*)d_W);
    } else {
        if (d_G) k_copy_rows<float><<<gr, 256, 0, ctx->st>>>(nc, nz, nb, lg, ctx->crow.as<int>(), ctx->G.as<cx<float>>(), (cx<float>*)d_G);
        if (d_W) k_copy_rows<float><<<gr, 256, 0, ctx->st>>>(nc, nz, nb, lw, ctx->crow.as<int>(), ctx->W.as<cx<float>>(), (cx<float>*)d_W);
    }
    MP3_CK(cudaGetLastError());
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_contract_multipoles(mp3pcf_ctx* ctx, double* d_upsilon, double* d_norm)
{
    if (!ctx || !d_upsilon || !d_norm) return fail(ctx, MP3PCF_EINVAL, "null argument");
    ctx->err.clear();
    const mp3pcf_config& c = ctx->cfg;
    const int64_t nc = ctx->n_centres;
    if (nc == 0) return MP3PCF_OK;
    const int nz = c.n_z, nb = c.n_bins;
    const int z3 = nz * nz * nz;
    const int groups = z3 * groups_per_zt(c.n_max);
    if (c.precision == MP3PCF_FP32_BF16X3 || c.precision == MP3PCF_FP32_TF32X3) {
        // tensor-core form: plan the centre slices, size the partials, launch, reduce
        const bool tf32 = c.precision == MP3PCF_FP32_TF32X3;
        ContractArgs<float> a{ctx->G.as<cx<float>>(), ctx->W.as<cx<float>>(), ctx->pay.as<Pay<float>>(),
                              ctx->zs.as<uint8_t>(), ctx->centre_idx.as<int>(), (int32_t)nc, nz, nb, c.n_max,
                              0, nullptr, nz > 1 ? ctx->zrange.as<int>() : nullptr};
        int splits = 0;
        unsigned long long* errw = ctx->pairs.as<unsigned long long>() + 1;
        MP3_CK(launch_contract_tc(a, tf32, ctx->n_sm, nullptr, errw, &splits, true, c.contract_slices, 0, ctx->st));
        MP3_CK(ctx->partial.ensure(sizeof(double) * 2 * (size_t)splits * groups * nb * nb));
        MP3_CK(ctx->ccoef.ensure(sizeof(float4) * (size_t)nc));
        a.splits = splits;
        a.partial = ctx->partial.as<double>();
        StageScope sc(ctx, ST_CONTRACT);
        ctx->launches[ST_CONTRACT] += 3;
        MP3_CK(launch_contract_tc(a, tf32, ctx->n_sm, ctx->ccoef.as<float4>(), errw, &splits, false,
                                  c.contract_slices, ctx->inject_wait_timeout ? 1 : 0, ctx->st));
        if (c.exclude_degenerate) {
            ctx->launches[ST_CONTRACT] += 1;
            MP3_CK(launch_contract_diag(a, ctx->st));
        }
        MP3_CK(launch_contract_reduce(ctx->partial.as<double>(), splits, nz, nb, c.n_max, d_upsilon, d_norm,
                                      ctx->st));
        if (c.exclude_degenerate) return degenerate_t<float>(ctx, d_upsilon, d_norm);
        return MP3PCF_OK;
    }
    int splits = (int)std::min<int64_t>(64, std::max<int64_t>(1, (int64_t)ctx->n_sm * 8 / groups));
    splits = (int)std::min<int64_t>(splits, std::max<int64_t>(1, nc / 256));
    MP3_CK(ctx->partial.ensure(sizeof(double) * 2 * (size_t)splits * groups * nb * nb));
    StageScope sc(ctx, ST_CONTRACT);
    ctx->launches[ST_CONTRACT] += 2;
    cudaError_t e;
    if (ctx->fp64) {
        ContractArgs<double> a{ctx->G.as<cx<double>>(), ctx->W.as<cx<double>>(), ctx->pay.as<Pay<double>>(),
                               ctx->zs.as<uint8_t>(),
                               ctx->centre_idx.as<int>(), (int32_t)nc, nz, nb, c.n_max, splits,
                               ctx->partial.as<double>(), nz > 1 ? ctx->zrange.as<int>() : nullptr};
        e = launch_contract_f64(a, ctx->st);
    } else {
        ContractArgs<float> a{ctx->G.as<cx<float>>(), ctx->W.as<cx<float>>(), ctx->pay.as<Pay<float>>(),
                              ctx->zs.as<uint8_t>(),
                              ctx->centre_idx.as<int>(), (int32_t)nc, nz, nb, c.n_max, splits,
                              ctx->partial.as<double>(), nz > 1 ? ctx->zrange.as<int>() : nullptr};
        e = launch_contract_f32(a, ctx->st);
    }
    MP3_CK(e);
    MP3_CK(launch_contract_reduce(ctx->partial.as<double>(), splits, nz, nb, c.n_max, d_upsilon, d_norm, ctx->st));
    if (c.exclude_degenerate)
        return ctx->fp64 ? degenerate_t<double>(ctx, d_upsilon, d_norm) : degenerate_t<float>(ctx, d_upsilon, d_norm);
    return MP3PCF_OK;
}

static PostArgs post_args(mp3pcf_ctx* ctx)
{
    const mp3pcf_config& c = ctx->cfg;
    PostArgs p;
    p.nz = c.n_z;
    p.nb = c.n_bins;
    p.n_max = c.n_max;
    p.n_phi = c.n_phi;
    p.norm_truncate = c.norm_truncate;
    p.edges = ctx->d_edges.as<double>();
    p.nodes = ctx->d_nodes.as<double>();
    return p;
}

mp3pcf_status mp3pcf_edge_correct(mp3pcf_ctx* ctx, const double* d_upsilon, const double* d_norm,
                                  double* d_gamma_n, int64_t* h_n_singular)
{
    if (!ctx || !d_upsilon || !d_norm || !d_gamma_n) return fail(ctx, MP3PCF_EINVAL, "null argument");
    ctx->err.clear();
    MP3_CK(cudaMemsetAsync(ctx->singular.p, 0, 8, ctx->st));
    {
        StageScope sc(ctx, ST_EDGE);
        ctx->launches[ST_EDGE] += 1;
        MP3_CK(launch_edge_correct(post_args(ctx), d_upsilon, d_norm, d_gamma_n,
                                   ctx->singular.as<unsigned long long>(), ctx->st));
    }
    if (h_n_singular) {
        unsigned long long ns = 0;
        MP3_CK(cudaMemcpyAsync(&ns, ctx->singular.p, 8, cudaMemcpyDeviceToHost, ctx->st));
        MP3_CK(cudaStreamSynchronize(ctx->st));
        *h_n_singular = (int64_t)ns;
        if (ns) return fail(ctx, MP3PCF_ESINGULAR, "singular mode-coupling systems");
    }
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_to_gamma(mp3pcf_ctx* ctx, const double* d_gamma_n, int32_t projection,
                              double* d_gamma_phi)
{
    if (!ctx || !d_gamma_n || !d_gamma_phi || projection < 0 || projection > 2)
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    StageScope sc(ctx, ST_GAMMA);
    ctx->launches[ST_GAMMA] += 1;
    MP3_CK(launch_to_gamma(post_args(ctx), d_gamma_n, projection, d_gamma_phi, ctx->st));
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_to_map3(mp3pcf_ctx* ctx, const double* d_gamma_cen, int64_t n_ap,
                             const double* d_theta_ap, double* d_corr, double* d_m8)
{
    if (!ctx || !d_gamma_cen || n_ap < 0 || n_ap > 65535 || (n_ap > 0 && (!d_theta_ap || (!d_corr && !d_m8))))
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    if (n_ap == 0) return MP3PCF_OK;
    const mp3pcf_config& c = ctx->cfg;
    const int z3 = c.n_z * c.n_z * c.n_z;
    const int chunks = 64;
    MP3_CK(ctx->m3partial.ensure(sizeof(double) * 8 * (size_t)z3 * n_ap * chunks));
    StageScope sc(ctx, ST_MAP3);
    ctx->launches[ST_MAP3] += 2;
    MP3_CK(launch_to_map3(post_args(ctx), d_gamma_cen, (int)n_ap, d_theta_ap,
                          ctx->m3partial.as<double>(), chunks, d_corr, d_m8, ctx->st));
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_to_map3_four(mp3pcf_ctx* ctx, const double* d_gamma_cen, int64_t n_ap, const double* d_theta_ap,
                                  double* d_m4)
{
    if (!ctx || !d_gamma_cen || n_ap < 0 || n_ap > 21845 || (n_ap > 0 && (!d_theta_ap || !d_m4)))
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    if (n_ap == 0) return MP3PCF_OK;
    const mp3pcf_config& c = ctx->cfg;
    const size_t z3 = (size_t)c.n_z * c.n_z * c.n_z;
    const int chunks = 64;
    MP3_CK(ctx->m3partial.ensure(sizeof(double) * 8 * z3 * 3 * n_ap * chunks));
    MP3_CK(ctx->m3four.ensure(sizeof(double) * (9 * (size_t)n_ap + 24 * z3 * n_ap)));
    StageScope sc(ctx, ST_MAP3);
    ctx->launches[ST_MAP3] += 4;
    double* theta3 = ctx->m3four.as<double>();
    MP3_CK(launch_to_map3_four(post_args(ctx), d_gamma_cen, (int)n_ap, d_theta_ap, theta3, theta3 + 9 * n_ap,
                               ctx->m3partial.as<double>(), chunks, d_m4, ctx->st));
    return MP3PCF_OK;
}

// ------------------------------------------------------------------ grid-based approximation

mp3pcf_status mp3pcf_grid_catalog(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq, const int32_t* d_yq,
                                  const float* d_g1, const float* d_g2, const float* d_w, const uint8_t* d_zbin,
                                  const int64_t* h_origin, int64_t pixel_q, int32_t npx, int32_t npy,
                                  int32_t* d_pxq, int32_t* d_pyq, float* d_pg1, float* d_pg2, float* d_pw,
                                  uint8_t* d_pzbin, int64_t* h_count)
{
    if (!ctx) return MP3PCF_EINVAL;
    const int nz = ctx->cfg.n_z;
    const int64_t npix = (int64_t)nz * npx * npy;
    if (n < 0 || !h_origin || pixel_q < 1 || npx < 1 || npy < 1 || npix > 0x7fffffffLL ||
        (n > 0 && (!d_xq || !d_yq || !d_g1 || !d_g2 || !d_w)) || !d_pxq || !d_pyq || !d_pg1 || !d_pg2 ||
        !d_pw || (nz > 1 && !d_pzbin) || !h_count)
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    // pixel centres must stay within the int32 fixed-point range
    const long long xmax = h_origin[0] + (long long)npx * pixel_q, ymax = h_origin[1] + (long long)npy * pixel_q;
    if (h_origin[0] < INT_MIN || h_origin[1] < INT_MIN || xmax > INT_MAX || ymax > INT_MAX)
        return fail(ctx, MP3PCF_EINVAL, "grid outside the fixed-point range");
    ctx->err.clear();
    MP3_CK(ctx->gridsum.ensure(sizeof(double) * 3 * (size_t)npix));
    MP3_CK(ctx->gridflag.ensure(sizeof(int) * 2 * ((size_t)npix + 1)));
    NvtxRange nvtx("mp3pcf grid_catalog");
    int* flags = ctx->gridflag.as<int>();
    int* rank = flags + npix + 1;
    MP3_CK(launch_grid_sums(n, d_xq, d_yq, d_g1, d_g2, d_w, d_zbin, nz, h_origin[0], h_origin[1], pixel_q, npx, npy,
                            ctx->gridsum.as<double>(), flags, ctx->n_sm, ctx->st));
    if (mp3pcf_status s = scan_exclusive(ctx, flags, rank, npix)) return s;
    MP3_CK(launch_grid_emit(nz, npx, npy, h_origin[0], h_origin[1], pixel_q, ctx->gridsum.as<double>(), rank, d_pxq,
                            d_pyq, d_pg1, d_pg2, d_pw, nz > 1 ? d_pzbin : nullptr, ctx->n_sm, ctx->st));
    int cnt = 0;
    MP3_CK(cudaMemcpyAsync(&cnt, rank + npix, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    MP3_CK(cudaStreamSynchronize(ctx->st));
    *h_count = cnt;
    return MP3PCF_OK;
}

// ------------------------------------------------------------------ direct estimator of <M_ap^3>

mp3pcf_status mp3pcf_map3_direct(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq, const int32_t* d_yq,
                                 const float* d_g1, const float* d_g2, const float* d_w, int64_t n_centres,
                                 const double* d_centres, int64_t n_ap, const double* d_theta_ap,
                                 double rcut_factor, double* d_out)
{
    if (!ctx) return MP3PCF_EINVAL;
    if (n < 0 || n_centres < 0 || n_ap < 0 || !(rcut_factor > 0.0) ||
        (n > 0 && (!d_xq || !d_yq || !d_g1 || !d_g2 || !d_w)) ||
        (n_centres > 0 && n_ap > 0 && (!d_centres || !d_theta_ap || !d_out)) ||
        n_centres * n_ap > 0x7fffffffLL)
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    if (n_centres == 0 || n_ap == 0) return MP3PCF_OK;
    NvtxRange nvtx("mp3pcf map3_direct");
    MP3_CK(launch_map3_direct(n, d_xq, d_yq, d_g1, d_g2, d_w, ctx->cfg.quantum, n_centres, d_centres, (int)n_ap,
                              d_theta_ap, rcut_factor, d_out, ctx->st));
    return MP3PCF_OK;
}

// ------------------------------------------------------------------ failure injection

mp3pcf_status mp3pcf_inject(mp3pcf_ctx* ctx, int32_t what, int32_t on)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->err.clear();
    switch (what) {
        case MP3PCF_INJECT_WAIT_TIMEOUT: ctx->inject_wait_timeout = on != 0; return MP3PCF_OK;
        case MP3PCF_INJECT_ALLOC_FAILURE: ctx->inject_alloc_failure = on != 0; return MP3PCF_OK;
        default: return fail(ctx, MP3PCF_EINVAL, "unknown injection");
    }
}

// ------------------------------------------------------------------ batching

mp3pcf_status mp3pcf_set_extent(mp3pcf_ctx* ctx, const int64_t* h_extent)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->err.clear();
    if (!h_extent) {
        ctx->fixed_extent = false;
        return MP3PCF_OK;
    }
    const int64_t x0 = h_extent[0], y0 = h_extent[1], x1 = h_extent[2], y1 = h_extent[3];
    if (x1 < x0 || y1 < y0 || x0 < INT_MIN || y0 < INT_MIN || x1 > INT_MAX || y1 > INT_MAX)
        return fail(ctx, MP3PCF_EINVAL, "bad extent");
    if (x1 - x0 >= (1LL << 24) || y1 - y0 >= (1LL << 24))
        return fail(ctx, MP3PCF_EINVAL, "patch extent must be below 2^24 position quanta");
    for (int i = 0; i < 4; ++i) ctx->ext[i] = h_extent[i];
    ctx->fixed_extent = true;
    return MP3PCF_OK;
}

// the whole path for one catalog of a batch into m8 (no host synchronisation)
static mp3pcf_status batch_one(mp3pcf_ctx* ctx, const mp3pcf_catalog_view& cv, int64_t n_ap, const double* theta,
                               double* m8)
{
    const mp3pcf_config& c = ctx->cfg;
    const size_t z3 = (size_t)c.n_z * c.n_z * c.n_z, nbb = (size_t)c.n_bins * c.n_bins;
    MP3_CK(cudaMemsetAsync(ctx->bups.p, 0, sizeof(double) * 2 * z3 * 4 * (c.n_max + 1) * nbb, ctx->st));
    MP3_CK(cudaMemsetAsync(ctx->bnorm.p, 0, sizeof(double) * 2 * z3 * (2 * c.n_max + 1) * nbb, ctx->st));
    mp3pcf_status s = mp3pcf_accumulate_moments(ctx, cv.n, cv.xq, cv.yq, cv.g1, cv.g2, cv.w, cv.zbin, nullptr);
    if (s == MP3PCF_OK) s = mp3pcf_contract_multipoles(ctx, ctx->bups.as<double>(), ctx->bnorm.as<double>());
    if (s == MP3PCF_OK)
        s = mp3pcf_edge_correct(ctx, ctx->bups.as<double>(), ctx->bnorm.as<double>(), ctx->bgam.as<double>(), nullptr);
    if (s == MP3PCF_OK) s = mp3pcf_to_gamma(ctx, ctx->bgam.as<double>(), 1, ctx->bgcen.as<double>());
    if (s == MP3PCF_OK) s = mp3pcf_to_map3(ctx, ctx->bgcen.as<double>(), n_ap, theta, nullptr, m8);
    if (s != MP3PCF_OK) return s;
    k_or_word<<<1, 32, 0, ctx->st>>>(ctx->pairs.as<unsigned long long>() + 1, ctx->berr.as<unsigned long long>());
    MP3_CK(cudaGetLastError());
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_run_batch(mp3pcf_ctx* ctx, const mp3pcf_catalog_view* h_cats, int64_t n_cats,
                               const int64_t* h_extent, int64_t n_ap, const double* d_theta_ap, double* d_m8,
                               int32_t use_graphs)
{
    NvtxRange nvtx_range("mp3pcf run_batch");
    if (!ctx || n_cats < 0 || (n_cats > 0 && (!h_cats || !h_extent || !d_m8)) || n_ap < 1 || n_ap > 65535 ||
        !d_theta_ap)
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    if (n_cats == 0) return MP3PCF_OK;
    for (int64_t i = 0; i < n_cats; ++i) {
        const mp3pcf_catalog_view& v = h_cats[i];
        if (v.n < 1 || v.n > INT_MAX / 2 || !v.xq || !v.yq || !v.g1 || !v.g2 || !v.w || (ctx->cfg.n_z > 1 && !v.zbin))
            return fail(ctx, MP3PCF_EINVAL, "bad catalog view");
    }
    const bool had_extent = ctx->fixed_extent;
    int64_t old_ext[4];
    for (int i = 0; i < 4; ++i) old_ext[i] = ctx->ext[i];
    if (mp3pcf_status s = mp3pcf_set_extent(ctx, h_extent)) return s;
    const bool had_timing = ctx->timing;
    ctx->timing = false;
    // the batch runs on a private non-blocking stream (the caller's may be the legacy default
    // stream, which cannot be captured), ordered after the caller's stream and before its next work
    if (!ctx->batch_st) {
        cudaError_t ec = cudaStreamCreateWithFlags(&ctx->batch_st, cudaStreamNonBlocking);
        for (int i = 0; ec == cudaSuccess && i < 2; ++i)
            ec = cudaEventCreateWithFlags(&ctx->batch_ev[i], cudaEventDisableTiming);
        if (ec != cudaSuccess) {
            ctx->timing = had_timing;
            ctx->fixed_extent = had_extent;
            for (int i = 0; i < 4; ++i) ctx->ext[i] = old_ext[i];
            return fail(ctx, MP3PCF_ECUDA, cudaGetErrorString(ec));
        }
    }
    cudaStream_t user_st = ctx->st;
    {
        cudaError_t ec = cudaEventRecord(ctx->batch_ev[0], user_st);
        if (ec == cudaSuccess) ec = cudaStreamWaitEvent(ctx->batch_st, ctx->batch_ev[0], 0);
        if (ec != cudaSuccess) {
            ctx->timing = had_timing;
            ctx->fixed_extent = had_extent;
            for (int i = 0; i < 4; ++i) ctx->ext[i] = old_ext[i];
            return fail(ctx, MP3PCF_ECUDA, cudaGetErrorString(ec));
        }
    }
    ctx->st = ctx->batch_st;
    const mp3pcf_config& c = ctx->cfg;
    const size_t z3 = (size_t)c.n_z * c.n_z * c.n_z, nbb = (size_t)c.n_bins * c.n_bins, D = 2 * c.n_max + 1;
    const size_t out_stride = z3 * (size_t)n_ap * 8;
    auto restore = [&](mp3pcf_status s) {
        if (cudaEventRecord(ctx->batch_ev[1], ctx->batch_st) == cudaSuccess)
            cudaStreamWaitEvent(user_st, ctx->batch_ev[1], 0);
        ctx->st = user_st;
        ctx->timing = had_timing;
        ctx->fixed_extent = had_extent;
        for (int i = 0; i < 4; ++i) ctx->ext[i] = old_ext[i];
        return s;
    };
    cudaError_t e;
    if ((e = ctx->bups.ensure(sizeof(double) * 2 * z3 * 4 * (c.n_max + 1) * nbb)) != cudaSuccess ||
        (e = ctx->bnorm.ensure(sizeof(double) * 2 * z3 * D * nbb)) != cudaSuccess ||
        (e = ctx->bgam.ensure(sizeof(double) * 2 * z3 * 4 * D * nbb)) != cudaSuccess ||
        (e = ctx->bgcen.ensure(sizeof(double) * 2 * z3 * 4 * nbb * c.n_phi)) != cudaSuccess ||
        (e = ctx->berr.ensure(16)) != cudaSuccess ||
        (e = cudaMemsetAsync(ctx->berr.p, 0, 16, ctx->st)) != cudaSuccess)
        return restore(fail(ctx, MP3PCF_ECUDA, cudaGetErrorString(e)));
    // the largest catalog runs first, uncaptured, so that every workspace buffer is at its final
    // size before any capture (a capture may not allocate)
    int64_t big = 0;
    for (int64_t i = 1; i < n_cats; ++i)
        if (h_cats[i].n > h_cats[big].n) big = i;
    if (mp3pcf_status s = batch_one(ctx, h_cats[big], n_ap, d_theta_ap, d_m8 + (size_t)big * out_stride))
        return restore(s);
    cudaGraphExec_t exec = nullptr;
    mp3pcf_status status = MP3PCF_OK;
    std::string capture_note;  // why a capture fell back to direct execution (first occurrence)
    for (int64_t i = 0; i < n_cats && status == MP3PCF_OK; ++i) {
        if (i == big) continue;
        double* out = d_m8 + (size_t)i * out_stride;
        if (!use_graphs) {
            status = batch_one(ctx, h_cats[i], n_ap, d_theta_ap, out);
            continue;
        }
        // capture the catalog's launches; the instantiated graph is updated in place when only
        // kernel parameters and grid sizes change (uneven galaxy counts), else re-instantiated
        cudaGraph_t graph = nullptr;
        cudaError_t eb = cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal);
        bool captured = eb == cudaSuccess;
        mp3pcf_status s = captured ? batch_one(ctx, h_cats[i], n_ap, d_theta_ap, out) : MP3PCF_ECUDA;
        const std::string during = s != MP3PCF_OK ? ctx->err : std::string();
        cudaError_t ee = captured ? cudaStreamEndCapture(ctx->st, &graph) : eb;
        if (captured && (ee != cudaSuccess || !graph)) captured = false;
        if (!captured || s != MP3PCF_OK) {
            if (capture_note.empty())
                capture_note = std::string("graph capture fell back to direct launches: ") +
                               (!during.empty() ? during : std::string(cudaGetErrorString(ee)));
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            status = batch_one(ctx, h_cats[i], n_ap, d_theta_ap, out);  // run it directly
            continue;
        }
        if (exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        }
        if (!exec) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess) ++ctx->graph_instantiations;
        }
        e = exec ? cudaGraphLaunch(exec, ctx->st) : cudaErrorUnknown;
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) status = fail(ctx, MP3PCF_ECUDA, cudaGetErrorString(e));
        else ++ctx->graph_launches;
    }
    unsigned long long berr = 0;
    e = cudaMemcpyAsync(&berr, ctx->berr.p, 8, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (exec) cudaGraphExecDestroy(exec);
    if (status != MP3PCF_OK) return restore(status);
    if (!capture_note.empty()) ctx->err = capture_note;  // not an error: the results are complete
    if (e != cudaSuccess) return restore(fail(ctx, MP3PCF_ECUDA, cudaGetErrorString(e)));
    if (berr & 4ULL) return restore(fail(ctx, MP3PCF_EINVAL, "a galaxy lies outside the extent or has zbin >= n_z"));
    if (berr) return restore(fail(ctx, MP3PCF_ETIMEOUT, "a bounded device wait gave up"));
    return restore(MP3PCF_OK);
}

mp3pcf_status mp3pcf_graph_stats(mp3pcf_ctx* ctx, int64_t* h_launches, int64_t* h_instantiations)
{
    if (!ctx) return MP3PCF_EINVAL;
    if (h_launches) *h_launches = ctx->graph_launches;
    if (h_instantiations) *h_instantiations = ctx->graph_instantiations;
    return MP3PCF_OK;
}

// ------------------------------------------------------------------ adjoints

mp3pcf_status mp3pcf_to_map3_adjoint(mp3pcf_ctx* ctx, int64_t n_ap, const double* d_theta_ap,
                                     const double* d_grad_corr, const double* d_grad_m8,
                                     double* d_grad_gamma_cen)
{
    if (!ctx || !d_grad_gamma_cen || n_ap < 0 || n_ap > 65535 || (n_ap > 0 && !d_theta_ap))
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    const mp3pcf_config& c = ctx->cfg;
    const size_t npts = (size_t)c.n_z * c.n_z * c.n_z * 4 * c.n_bins * c.n_bins * c.n_phi;
    if (n_ap == 0 || (!d_grad_corr && !d_grad_m8)) {
        MP3_CK(cudaMemsetAsync(d_grad_gamma_cen, 0, sizeof(double) * 2 * npts, ctx->st));
        return MP3PCF_OK;
    }
    StageScope sc(ctx, ST_MAP3);
    ctx->launches[ST_MAP3] += 1;
    MP3_CK(launch_to_map3_adjoint(post_args(ctx), (int)n_ap, d_theta_ap, d_grad_corr, d_grad_m8,
                                  d_grad_gamma_cen, ctx->st));
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_to_gamma_adjoint(mp3pcf_ctx* ctx, int32_t projection, const double* d_grad_gamma_phi,
                                      double* d_grad_gamma_n)
{
    if (!ctx || !d_grad_gamma_phi || !d_grad_gamma_n || (projection != 0 && projection != 1))
        return fail(ctx, MP3PCF_EINVAL, "bad argument");
    ctx->err.clear();
    StageScope sc(ctx, ST_GAMMA);
    ctx->launches[ST_GAMMA] += 1;
    MP3_CK(launch_to_gamma_adjoint(post_args(ctx), d_grad_gamma_phi, projection, d_grad_gamma_n, ctx->st));
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_edge_correct_adjoint(mp3pcf_ctx* ctx, const double* d_norm, const double* d_gamma_n,
                                          const double* d_grad_gamma_n, double* d_grad_upsilon,
                                          double* d_grad_norm)
{
    if (!ctx || !d_norm || !d_gamma_n || !d_grad_gamma_n || !d_grad_upsilon || !d_grad_norm)
        return fail(ctx, MP3PCF_EINVAL, "null argument");
    ctx->err.clear();
    const PostArgs p = post_args(ctx);
    MP3_CK(ctx->adjscratch.ensure(edge_correct_adjoint_scratch(p)));
    StageScope sc(ctx, ST_EDGE);
    ctx->launches[ST_EDGE] += 2;
    MP3_CK(launch_edge_correct_adjoint(p, d_norm, d_gamma_n, d_grad_gamma_n, ctx->adjscratch.as<double>(),
                                       d_grad_upsilon, d_grad_norm, ctx->st));
    return MP3PCF_OK;
}

}  // extern "C"

// the catalog state of the last accumulate call as AdjArgs (gradient buffers left null)
template <typename T>
static AdjArgs<T> catalog_args(mp3pcf_ctx* ctx)
{
    const mp3pcf_config& c = ctx->cfg;
    AdjArgs<T> a{};
    a.n_centres = (int32_t)ctx->n_centres;
    a.nz = c.n_z;
    a.nb = c.n_bins;
    a.n_max = c.n_max;
    a.centre_idx = ctx->centre_idx.as<int>();
    a.pos = ctx->pos.as<int2>();
    a.pay = ctx->pay.as<Pay<T>>();
    a.zs = c.n_z > 1 ? ctx->zs.as<uint8_t>() : nullptr;
    a.cell_start = ctx->count.as<int>();
    a.g = ctx->grid;
    a.e2q = ctx->d_e2q.as<long long>();
    a.G = ctx->G.as<cx<T>>();
    a.W = ctx->W.as<cx<T>>();
    return a;
}

template <typename T>
static mp3pcf_status degenerate_t(mp3pcf_ctx* ctx, double* ups, double* norm)
{
    const mp3pcf_config& c = ctx->cfg;
    MP3_CK(ctx->degen.ensure(sizeof(cx<T>) * 4 * (size_t)ctx->n_centres * c.n_z * c.n_bins));
    ctx->launches[ST_CONTRACT] += 2;
    const AdjArgs<T> a = catalog_args<T>(ctx);
    if constexpr (sizeof(T) == 8)
        MP3_CK(launch_degenerate_f64(a, ctx->degen.p, ups, norm, ctx->n_sm, ctx->st));
    else
        MP3_CK(launch_degenerate_f32(a, ctx->degen.p, ups, norm, ctx->n_sm, ctx->st));
    return MP3PCF_OK;
}

template <typename T>
static mp3pcf_status moments_adjoint_t(mp3pcf_ctx* ctx, const double* gups, const double* gnorm, const float* g1,
                                       const float* g2, const float* w, float* dg1, float* dg2, float* dw)
{
    const mp3pcf_config& c = ctx->cfg;
    const int64_t n = ctx->n, nc = ctx->n_centres;
    const int nz = c.n_z, nb = c.n_bins;
    MP3_CK(ctx->gv.ensure(sizeof(T) * 4 * (size_t)std::max<int64_t>(n, 1)));
    const size_t ngroups = (size_t)nz * nz * nz * (4 * (c.n_max + 1) + 2 * c.n_max + 1);
    MP3_CK(ctx->gtab.ensure(2 * sizeof(cx<T>) * ngroups * nb * nb));
    if (nc > 0) {
        MP3_CK(ctx->gG.ensure(sizeof(cx<T>) * (size_t)(2 * c.n_max + 3) * nc * nz * nb_pad(nb)));
        MP3_CK(ctx->gW.ensure(sizeof(cx<T>) * (size_t)(2 * c.n_max + 1) * nc * nz * nb_pad(nb)));
    }
    AdjArgs<T> a;
    a.n_centres = (int32_t)nc;
    a.nz = nz;
    a.nb = nb;
    a.n_max = c.n_max;
    a.centre_idx = ctx->centre_idx.as<int>();
    a.pos = ctx->pos.as<int2>();
    a.pay = ctx->pay.as<Pay<T>>();
    a.zs = nz > 1 ? ctx->zs.as<uint8_t>() : nullptr;
    a.cell_start = ctx->count.as<int>();
    a.g = ctx->grid;
    a.e2q = ctx->d_e2q.as<long long>();
    a.G = ctx->G.as<cx<T>>();
    a.W = ctx->W.as<cx<T>>();
    a.gups = gups;
    a.gnorm = gnorm;
    a.gG = ctx->gG.as<cx<T>>();
    a.gW = ctx->gW.as<cx<T>>();
    a.gvw = ctx->gv.as<T>();
    a.dgs = nullptr;
    if (c.exclude_degenerate) {
        MP3_CK(ctx->degen_grad.ensure(sizeof(cx<double>) * 4 * (size_t)nz * nz * nb));
        a.dgs = ctx->degen_grad.as<cx<double>>();
    }
    a.tabX = ctx->gtab.as<cx<T>>();
    a.tabY = a.tabX + ngroups * nb * nb;
    StageScope sc(ctx, ST_MOMENTS);
    ctx->launches[ST_MOMENTS] += nc > 0 ? 4 : 1;
    cudaError_t e;
    if constexpr (sizeof(T) == 8)
        e = launch_moments_adjoint_f64(a, n, ctx->perm.as<int>(), g1, g2, w, dg1, dg2, dw, ctx->n_sm, ctx->st);
    else
        e = launch_moments_adjoint_f32(a, n, ctx->perm.as<int>(), g1, g2, w, dg1, dg2, dw, ctx->n_sm, ctx->st);
    MP3_CK(e);
    return MP3PCF_OK;
}

extern "C" {

mp3pcf_status mp3pcf_moments_adjoint(mp3pcf_ctx* ctx, const double* d_grad_upsilon, const double* d_grad_norm,
                                     int64_t n, const float* d_g1, const float* d_g2, const float* d_w,
                                     float* d_grad_g1, float* d_grad_g2, float* d_grad_w)
{
    NvtxRange nvtx_range("mp3pcf moments_adjoint");
    if (!ctx || !d_grad_upsilon || !d_grad_norm) return fail(ctx, MP3PCF_EINVAL, "null argument");
    ctx->err.clear();
    if (n != ctx->n) return fail(ctx, MP3PCF_EINVAL, "n differs from the last accumulate call");
    if (ctx->combined) return fail(ctx, MP3PCF_EUNSUPPORTED, "no adjoint of the combined estimator's grid bins");
    if (n == 0) return MP3PCF_OK;
    if (!d_g1 || !d_g2 || !d_w) return fail(ctx, MP3PCF_EINVAL, "null catalog pointer");
    if (ctx->fp64) return moments_adjoint_t<double>(ctx, d_grad_upsilon, d_grad_norm, d_g1, d_g2, d_w, d_grad_g1,
                                                    d_grad_g2, d_grad_w);
    return moments_adjoint_t<float>(ctx, d_grad_upsilon, d_grad_norm, d_g1, d_g2, d_w, d_grad_g1, d_grad_g2,
                                    d_grad_w);
}

mp3pcf_status mp3pcf_set_timing(mp3pcf_ctx* ctx, int32_t on)
{
    if (!ctx) return MP3PCF_EINVAL;
    ctx->timing = on != 0;
    return MP3PCF_OK;
}

mp3pcf_status mp3pcf_stage_times(mp3pcf_ctx* ctx, double* h_ms, int64_t* h_launches, int32_t reset)
{
    if (!ctx) return MP3PCF_EINVAL;
    MP3_CK(cudaStreamSynchronize(ctx->st));
    double ms[6] = {0, 0, 0, 0, 0, 0};
    for (auto& pr : ctx->ev) {
        float t = 0.f;
        MP3_CK(cudaEventElapsedTime(&t, pr.second.first, pr.second.second));
        ms[pr.first] += t;
    }
    for (int i = 0; i < 6; ++i) {
        if (h_ms) h_ms[i] = ms[i];
        if (h_launches) h_launches[i] = ctx->launches[i];
    }
    if (reset) {
        for (auto& pr : ctx->ev) {
            ctx->pool.push_back(pr.second.first);
            ctx->pool.push_back(pr.second.second);
        }
        ctx->ev.clear();
        for (int i = 0; i < 6; ++i) ctx->launches[i] = 0;
    }
    return MP3PCF_OK;
}

}  // extern "C"
