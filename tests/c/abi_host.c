/* A plain C99 caller of the C ABI: includes only include/mp3pcf.h and links libmp3pcf.so. It makes
 * host-only calls (no GPU needed): the bin-edge table of a valid configuration, which it prints,
 * and the argument checks that return before any CUDA call. Exit status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "mp3pcf.h"

static int failures = 0;

static void check(int ok, const char* what)
{
    if (!ok) {
        fprintf(stderr, "FAILED: %s\n", what);
        ++failures;
    }
}

int main(void)
{
    mp3pcf_config cfg;
    double edges[21];
    int64_t edges2[21];
    mp3pcf_ctx* ctx = NULL;
    int b;

    memset(&cfg, 0, sizeof cfg);
    cfg.n_bins = 20;
    cfg.theta_min = 0.5;
    cfg.theta_max = 120.0;
    cfg.n_max = 30;
    cfg.n_phi = 100;
    cfg.n_z = 1;
    cfg.quantum = 1.0 / 8192.0;
    cfg.precision = MP3PCF_FP32_BF16X3;

    check(mp3pcf_bin_edges(&cfg, edges, edges2) == MP3PCF_OK, "bin edges of a valid configuration");
    for (b = 0; b <= cfg.n_bins; ++b) printf("%d %.17g %lld\n", b, edges[b], (long long)edges2[b]);
    for (b = 0; b < cfg.n_bins; ++b) check(edges[b] < edges[b + 1] && edges2[b] < edges2[b + 1], "increasing");

    cfg.n_bins = 0;
    check(mp3pcf_create(&cfg, NULL, &ctx) == MP3PCF_EINVAL && ctx == NULL, "bad configuration refused");
    check(mp3pcf_bin_edges(&cfg, NULL, NULL) == MP3PCF_EINVAL, "bad configuration: no edges");
    check(mp3pcf_create(NULL, NULL, &ctx) == MP3PCF_EINVAL, "null configuration refused");
    check(mp3pcf_destroy(NULL) == MP3PCF_OK, "destroy(NULL)");
    check(mp3pcf_last_error(NULL) != NULL, "last_error(NULL) is a string");
    return failures == 0 ? 0 : 1;
}
