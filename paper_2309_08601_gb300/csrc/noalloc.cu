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

// device address of the scratch array, looked up once per device
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {nullptr};

static cudaError_t noalloc_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
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
    if (!d_gamma_cen || n_ap < 0 || (n_ap > 0 && !d_theta_ap)) return MP3PCF_EINVAL;
    const int nb = cfg->n_bins;
    const long long jobs = (long long)cfg->n_z * cfg->n_z * cfg->n_z * n_ap;
    if (jobs > (long long)kNoAllocMaxJobs) return MP3PCF_EINVAL;  // beyond the static scratch
    if (n_ap == 0) return MP3PCF_OK;
    for (int b = 0; b < nb; ++b)
        t.nodes[b] = cfg->radial_nodes ? sqrt(t.e[b] * t.e[b + 1]) : 0.5 * (t.e[b] + t.e[b + 1]);
    double* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return MP3PCF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
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
