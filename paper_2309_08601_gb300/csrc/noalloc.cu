// Allocation-free variant of the aperture-measure step (mp3pcf_to_map3_noalloc).
//
// Some callers cannot allocate device memory: a plugin running inside a host application that
// owns every byte of device memory through its own pool, or a service that must keep a fixed
// memory budget and may not call cudaMalloc (which can also synchronise the device) while it
// is serving. This entry point needs no context and allocates nothing. Its only scratch, the
// per-block partial sums of the quadrature and the small tables of bin edges and nodes, lives
// in one file-scope device array that every GPU loading the library holds until the process
// exits.
#include <mutex>

#include "common.cuh"

namespace mp3 {

// 1 MiB of scratch: the edge table, the node table and the partial sums of at most
// kNoAllocMaxJobs (Z-triplet, aperture) jobs.
constexpr int kNoAllocChunks = 64;                 // blocks per job, as in mp3pcf_to_map3
constexpr size_t kNoAllocDoubles = 131072;         // 1 MiB
constexpr size_t kNoAllocTables = 256;             // doubles reserved for edges and nodes
constexpr size_t kNoAllocMaxJobs = (kNoAllocDoubles - kNoAllocTables) / (8 * kNoAllocChunks);

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

struct NoAllocTables {
    double e[kMaxBins + 1];
    double nodes[kMaxBins];
};

__global__ void noalloc_write_tables(const NoAllocTables t, int nb, double* dst)
{
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) dst[i] = t.e[i];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) dst[kMaxBins + 1 + i] = t.nodes[i];
}

// Device address of the scratch array. It belongs to the module the runtime loaded into the
// current context, so it is cached per context (the driver's context handle, obtained through the
// runtime's driver entry point, needs no link to libcuda). Outside stream capture every call looks
// the address up again and refreshes the cache: after cudaDeviceReset the module is loaded anew
// and the array may have moved, and a non-primary context has its own copy. During capture the
// lookup (which may load the module) is not attempted and the cached address of the current
// context is used; without one the call fails.
typedef int (*CtxGetCurrentFn)(void**);

static std::mutex g_noalloc_mu;
constexpr int kNoAllocCtxSlots = 64;
static void* g_noalloc_ctx[kNoAllocCtxSlots] = {nullptr};
static double* g_noalloc_ptr[kNoAllocCtxSlots] = {nullptr};
static int g_noalloc_next = 0;

static void* current_context()
{
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

static cudaError_t noalloc_scratch(cudaStream_t st, double** out)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    void* ctx = current_context();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    int slot = -1;
    for (int i = 0; i < kNoAllocCtxSlots; ++i)
        if (g_noalloc_ptr[i] && g_noalloc_ctx[i] == ctx) slot = i;
    if (cap != cudaStreamCaptureStatusNone) {
        if (slot < 0 || !ctx) return cudaErrorStreamCaptureUnsupported;
        *out = g_noalloc_ptr[slot];
        return cudaSuccess;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (ctx) {
        if (slot < 0) {
            slot = g_noalloc_next;
            g_noalloc_next = (g_noalloc_next + 1) % kNoAllocCtxSlots;
        }
        g_noalloc_ctx[slot] = ctx;
        g_noalloc_ptr[slot] = static_cast<double*>(p);
    }
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace mp3

using namespace mp3;

extern "C" mp3pcf_status mp3pcf_to_map3_noalloc(const mp3pcf_config* cfg, void* stream,
                                                 const double* d_gamma_cen, int64_t n_ap,
                                                 const double* d_theta_ap, double* d_corr,
                                                 double* d_m8)
{
    NoAllocTables t;
    if (!cfg || mp3pcf_bin_edges(cfg, t.e, nullptr) != MP3PCF_OK) return MP3PCF_EINVAL;
    if (!d_gamma_cen || n_ap < 0 || (n_ap > 0 && (!d_theta_ap || (!d_corr && !d_m8)))) return MP3PCF_EINVAL;
    const int nb = cfg->n_bins;
    const long long jobs = (long long)cfg->n_z * cfg->n_z * cfg->n_z * n_ap;
    if (jobs > (long long)kNoAllocMaxJobs) return MP3PCF_EINVAL;  // beyond the static scratch
    if (n_ap == 0) return MP3PCF_OK;
    for (int b = 0; b < nb; ++b)
        t.nodes[b] = cfg->radial_nodes ? sqrt(t.e[b] * t.e[b + 1]) : 0.5 * (t.e[b] + t.e[b + 1]);
    double* scratch = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (noalloc_scratch(st, &scratch) != cudaSuccess) return MP3PCF_ECUDA;
    noalloc_write_tables<<<1, 128, 0, st>>>(t, nb, scratch);
    if (cudaGetLastError() != cudaSuccess) return MP3PCF_ECUDA;
    PostArgs p;
    p.nz = cfg->n_z;
    p.nb = nb;
    p.n_max = cfg->n_max;
    p.n_phi = cfg->n_phi;
    p.norm_truncate = cfg->norm_truncate;
    p.edges = scratch;
    p.nodes = scratch + kMaxBins + 1;
    if (launch_to_map3(p, d_gamma_cen, (int)n_ap, d_theta_ap, scratch + kNoAllocTables,
                       kNoAllocChunks, d_corr, d_m8, st) != cudaSuccess)
        return MP3PCF_ECUDA;
    return MP3PCF_OK;
}
