/*
 * mp3pcf — GB300 (sm_103a) library for the multipole estimator of the shear three-point
 * correlation function of Porth et al. (2023), "Efficient estimation of third-order shear
 * correlation functions".
 *
 * C ABI. All pointers named d_* are DEVICE pointers owned by the caller; all pointers named
 * h_* are HOST pointers owned by the caller. The context owns only its own workspace. Every
 * call is stream-ordered on the stream given to mp3pcf_create and returns a status code; no
 * call throws. Calls that must return a count to the host (noted below) synchronise the stream.
 * One context must not be used from two host threads at the same time.
 *
 * Complex numbers are interleaved (re, im). Floating-point outputs of the multipole stages are
 * always FP64; the moments are FP32 or FP64 as the precision setting says.
 *
 * Conventions (Sec. 2 and Sec. 3 of the paper):
 *   gamma_c = gamma_1 + i gamma_2; a galaxy's contribution carries v = w gamma_c;
 *   radial bins are logarithmic, e_b = theta_min (theta_max/theta_min)^(b/n_bins), b = 0..n_bins,
 *   and a pair is in bin b iff e_b <= separation < e_{b+1}; the test is exact, on the integer
 *   squared separation of the fixed-point positions against ceil((e_b/quantum)^2);
 *   Z-triplet index zt = (Z1*n_z + Z2)*n_z + Z3 (centre galaxy in Z1, the galaxy at the first
 *   radial bin in Z2, the one at the second radial bin in Z3), Eq. tomoGn.
 */
#ifndef MP3PCF_H
#define MP3PCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MP3PCF_OK = 0,
    MP3PCF_EINVAL = 1,      /* bad argument or configuration */
    MP3PCF_ENOMEM = 2,      /* device workspace could not be allocated */
    MP3PCF_ECUDA = 3,       /* a CUDA runtime call failed; see mp3pcf_last_error */
    MP3PCF_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    MP3PCF_ESINGULAR = 5,   /* at least one mode-coupling system was singular (N_0 = 0) */
    MP3PCF_EUNSUPPORTED = 6 /* valid request this build does not implement */
} mp3pcf_status;

typedef enum {
    MP3PCF_FP64 = 0,        /* moments and contraction in FP64 */
    MP3PCF_FP32 = 1,        /* moments in FP32, contraction FP32 with FP64 tile sums */
    MP3PCF_FP32_BF16X3 = 2, /* moments in FP32, contraction on tensor cores, BF16 hi+lo split */
    MP3PCF_FP32_TF32X3 = 3  /* moments in FP32, contraction on tensor cores, TF32 hi+lo split */
} mp3pcf_precision;

typedef struct {
    int32_t n_bins;        /* number of logarithmic radial bins, >= 1 */
    double theta_min;      /* inner edge of the first bin, arcmin, > 0 */
    double theta_max;      /* outer edge of the last bin, arcmin, > theta_min */
    int32_t n_max;         /* largest multipole order, 0 <= n_max <= 50 */
    int32_t n_phi;         /* angular grid of to_gamma/to_map3, phi_k = (k+1/2) 2 pi/n_phi */
    int32_t n_z;           /* tomographic bins, 1..8 (1 = no tomography) */
    double quantum;        /* arcmin per unit of the int32 fixed-point positions, > 0 */
    int32_t precision;     /* mp3pcf_precision */
    int32_t norm_truncate; /* 1: drop N_m with |m| > n_max from the coupling matrix */
    int32_t radial_nodes;  /* 0: bin node (e_b+e_{b+1})/2, 1: sqrt(e_b e_{b+1}) */
    int32_t cell_occupancy;  /* tile shape of the moment kernel: target galaxies per grid cell and
                              * redshift bin, 0 = default (4), else 1..64 (an autotuner picks it) */
    int32_t contract_slices; /* slices of the centre axis in the tensor-core contraction, 0 = auto
                              * (whole waves of resident CTAs), else 1..64 */
    int32_t exclude_degenerate; /* 1: leave the triplets with j = k (one neighbour in both legs, so
                                 * b1 = b2 and Z2 = Z3) out of Upsilon and N; 0 (default): the
                                 * paper's sums over all (i, j, k) */
    int32_t grid_fft;        /* combined estimator (mp3pcf_accumulate_moments_combined): 1 evaluates
                              * the grid levels' moments by FFT convolution of the gridded fields with
                              * the bin kernels (Sec. 3.2), 0 (default) by direct sums over pixel pairs;
                              * the two agree to the FFT's rounding */
    int32_t reserved;        /* must be zero */
} mp3pcf_config;

typedef struct mp3pcf_ctx mp3pcf_ctx;

/* Validates cfg, binds the current CUDA device and the given stream (cudaStream_t, may be
 * NULL for the legacy default stream), and creates a context. On success *out owns the context;
 * release it with mp3pcf_destroy. EINVAL on a bad configuration (nothing is allocated). */
mp3pcf_status mp3pcf_create(const mp3pcf_config* cfg, void* stream, mp3pcf_ctx** out);

/* Frees the context and its workspace (synchronises its stream). NULL is accepted. */
mp3pcf_status mp3pcf_destroy(mp3pcf_ctx* ctx);

/* Text of the last error on this context (never NULL; empty if none). */
const char* mp3pcf_last_error(const mp3pcf_ctx* ctx);

/* Host-only, no CUDA call: the bin edges e_b (arcmin, n_bins+1 values) and the exact integer
 * squared edges ceil((e_b/quantum)^2) (n_bins+1 values) the pair test uses (Sec. 2.4; the
 * half-open reading of the bin interval). Either output may be NULL. */
mp3pcf_status mp3pcf_bin_edges(const mp3pcf_config* cfg, double* h_edges, int64_t* h_edges2_q);

/* Stage (a), Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization, Sec. 3.1. For every selected
 * centre galaxy i, radial bin b and neighbour bin Z:
 *   G_m(i,b,Z) = sum_k w_k gamma_c,k e^{i m varphi_ik} [theta_ik in bin b, zbin_k = Z],
 *                m = -n_max-3 .. n_max-1,
 *   W_m(i,b,Z) = sum_k w_k e^{i m varphi_ik} [...],  m = 0 .. 2 n_max,
 * over all n galaxies k as neighbours. Inputs (device, n entries each): d_xq, d_yq int32
 * fixed-point positions (units of cfg.quantum; differences must fit in int32), d_g1, d_g2, d_w
 * float32 (w >= 0), d_zbin uint8 in [0, n_z) or NULL (all bin 0), d_centre_mask uint8 or NULL
 * (NULL: every galaxy is a centre; else galaxy i is a centre iff mask[i] != 0). The catalog is
 * cell-sorted into the context's workspace; results stay in the context (read them with
 * mp3pcf_copy_moments, contract them with mp3pcf_contract_multipoles). n = 0 is allowed.
 * Synchronises the stream once (grid extent and centre count). */
mp3pcf_status mp3pcf_accumulate_moments(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq,
                                        const int32_t* d_yq, const float* d_g1, const float* d_g2,
                                        const float* d_w, const uint8_t* d_zbin,
                                        const uint8_t* d_centre_mask);

/* Number of centres of the last accumulate call and the number of ordered (centre, neighbour)
 * pairs it accumulated (host outputs, either may be NULL). Synchronises the stream. Returns
 * ETIMEOUT if a bounded device-side wait of the moment kernel, or of a tensor-core contraction
 * launched since that accumulate call, gave up (their outputs are then invalid). */
mp3pcf_status mp3pcf_counts(mp3pcf_ctx* ctx, int64_t* h_n_centres, int64_t* h_n_pairs);

/* Copies the moments of the last accumulate call to caller device buffers, centres in
 * increasing galaxy index: d_G [n_centres][n_z][n_bins][2 n_max + 3] (m = -n_max-3..n_max-1),
 * d_W [n_centres][n_z][n_bins][2 n_max + 1] (m = 0..2 n_max), complex float for the FP32 modes
 * and complex double for MP3PCF_FP64. Either pointer may be NULL. */
mp3pcf_status mp3pcf_copy_moments(mp3pcf_ctx* ctx, void* d_G, void* d_W);

/* Stage (b), Eqs. Upsilon0_Derivation, Upsilon1-3, 3PCF_Normalization and tomoGn, Sec. 3.1:
 *   Upsilon_0,n = - sum_i v_i   G_{n-3}(b1) G_{-n-3}(b2)
 *   Upsilon_1,n = - sum_i v_i^* G_{n-1}(b1) G_{-n-1}(b2)
 *   Upsilon_2,n = - sum_i v_i   G_{-n-1}(b1)^* G_{-n-3}(b2)
 *   Upsilon_3,n = - sum_i v_i   G_{n-3}(b1) G_{n-1}(b2)^*
 *   N_n         =   sum_i w_i   W_n(b1) W_n(b2)^*
 * summed over the centres of the last accumulate call and ADDED to d_upsilon
 * [n_z^3][4][n_max+1][n_bins][n_bins] (n = 0..n_max) and d_norm [n_z^3][2 n_max+1][n_bins][n_bins]
 * (n = 0..2 n_max), complex double. Adding lets callers sum centre chunks or patches
 * (App. B, Eq. PatchGamma). With exclude_degenerate the j = k triplets of these centres are
 * removed: for b1 = b2 and Z2 = Z3, Upsilon_0 += sum_i v_i sum_k v_k^2 e^{-6i phi_ik},
 * Upsilon_1 += sum_i v_i^* sum_k v_k^2 e^{-2i phi}, Upsilon_2,3 += sum_i v_i sum_k |v_k|^2
 * e^{-2i phi} and N -= sum_i w_i sum_k w_k^2 (v = w gamma), for every order.
 * MP3PCF_FP64 and MP3PCF_FP32 sum on the CUDA cores (tile sums in the moment precision, added in
 * FP64). MP3PCF_FP32_BF16X3 / MP3PCF_FP32_TF32X3 run the components as real GEMMs over the
 * centres on the tcgen05 tensor cores (Upsilon_0..3 of one order share a tile and its four moment
 * rows): every FP32 operand x = hi + lo (hi, lo in BF16 resp. TF32), products
 * hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory over chains of 512 (256) centres,
 * the chains added in FP32 per centre slice and the slices in FP64 in a fixed order. A bounded
 * wait that gives up in that kernel is reported as ETIMEOUT by the next mp3pcf_counts. */
mp3pcf_status mp3pcf_contract_multipoles(mp3pcf_ctx* ctx, double* d_upsilon, double* d_norm);

/* Edge correction, Eqs. ModeCoupling and GammaMultipolesWithEC, Sec. 3.4: per (zt, b1, b2)
 * solves sum_n N_{l-n} Gamma_{mu,n} = Upsilon_{mu,l}, l, n in [-n_max, n_max], in FP64 with
 * partial pivoting. Negative orders come from the symmetries of App. A
 * (Upsilon_{0,-n}(i,j) = Upsilon_{0,n}(j,i), Upsilon_{1,-n}(i,j) = Upsilon_{1,n}(j,i),
 * Upsilon_{2,-n}(i,j) = Upsilon_{3,n}(j,i), N_{-n}(i,j) = N_n(j,i), with Z2 <-> Z3).
 * Output d_gamma_n [n_z^3][4][2 n_max+1][n_bins][n_bins] complex double, n = -n_max..n_max;
 * Gamma(phi) = sum_n Gamma_n e^{i n phi} (no 1/2pi, the normalisation Eq. ModeCoupling
 * implies). Systems with N_0 = 0 or a zero pivot get NaN and the call returns ESINGULAR with
 * their number in *h_n_singular (host, may be NULL; a non-NULL pointer synchronises). */
mp3pcf_status mp3pcf_edge_correct(mp3pcf_ctx* ctx, const double* d_upsilon, const double* d_norm,
                                  double* d_gamma_n, int64_t* h_n_singular);

/* Gamma^x_mu(b1, b2, phi_k) = sum_n Gamma_{mu,n} e^{i n phi_k}, phi_k = (k+1/2) 2 pi / n_phi
 * (Sec. 4: linear angular bins on [0, 2 pi]); projection 1 multiplies by the rotation factors
 * of Eqs. X2Centroid0-3 (Sec. 2.3) evaluated at the radial nodes of b1 and b2, giving the
 * centroid projection; projection 2 is the x-projection averaged over each angular bin
 * [phi_k - pi/n_phi, phi_k + pi/n_phi) (each term times sinc(n pi / n_phi)), the binned
 * estimate of Sec. 2.4 (Eq. Gamma0_binned) that angular-bin sums of triplets compare with.
 * Output d_gamma_phi [n_z^3][4][n_bins][n_bins][n_phi] complex double. */
mp3pcf_status mp3pcf_to_gamma(mp3pcf_ctx* ctx, const double* d_gamma_n, int32_t projection,
                              double* d_gamma_phi);

/* Third-order aperture measures, Eqs. MFrom3pcfTheory, MFrom3pcfTheoryb (Sec. 5.2) with the
 * Q filter of Eq. CrittendenQ and the filters of App. C, by the midpoint rule over the radial
 * bins and the n_phi angular nodes:
 *   corr_mu = sum_{b1,b2,k} Gamma^cen_mu(b1,b2,phi_k) F_mu(t_b1, t_b2, phi_k) dt_b1 dt_b2 dphi.
 * d_gamma_cen: output of mp3pcf_to_gamma with projection 1. d_theta_ap [n_ap][3] aperture radii
 * (arcmin, device). Outputs (device): d_corr [n_z^3][n_ap][4] complex double
 * (<M^3>, <M^* M^2>, <M M^* M>, <M^2 M^*>) and d_m8 [n_z^3][n_ap][8] double, the eight real
 * measures of Eqs. MapTrafo8_1-8 in the order Map^3, <Mx Map Map>, <Map Mx Map>,
 * <Map Map Mx>, <Map Mx Mx>, <Mx Map Mx>, <Mx Mx Map>, Mx^3. Either output may be NULL, not both
 * (EINVAL when n_ap > 0). */
mp3pcf_status mp3pcf_to_map3(mp3pcf_ctx* ctx, const double* d_gamma_cen, int64_t n_ap,
                             const double* d_theta_ap, double* d_corr, double* d_m8);

/* The shorter four-equation form of the aperture measures (App. C, Eqs. MapTrafo4_1-4), a
 * cross-check of the eight-equation form: from <M^3>(t1,t2,t3) and the one-conjugate correlator
 * at three orderings of the radii. The printed equations place the conjugate on the last radius of
 * each ordering; this library's <M^* M^2> (Gamma_1 with F_1) conjugates the first, so they are
 * evaluated at (t3,t1,t2), (t2,t1,t3) and (t1,t2,t3). Output d_m4 [n_z^3][n_ap][4] double:
 * Map^3, <Map Map Mx>, <Map Mx Mx>, Mx^3 at (t1,t2,t3). It agrees with mp3pcf_to_map3 where the
 * estimated correlators obey the relabelling symmetries the appendix uses (to the quadrature and
 * binning of the 3PCF). n_ap <= 21845; the context holds the scratch. */
mp3pcf_status mp3pcf_to_map3_four(mp3pcf_ctx* ctx, const double* d_gamma_cen, int64_t n_ap,
                                  const double* d_theta_ap, double* d_m4);

/* ---- Grid-based approximation (Sec. 3.2): the pixel catalog of a regular grid. Pixel (ix, iy)
 * of z-bin z covers [origin[0] + ix * pixel_q, origin[0] + (ix + 1) * pixel_q) x (the same in y),
 * in fixed-point quanta; galaxies outside the grid count in its edge pixels. Each non-empty pixel
 * becomes a galaxy at its centre (origin + i * pixel_q + pixel_q / 2) with weight W = sum of w and
 * shear (sum of w gamma) / W, written in (z, iy, ix) order to the caller's device arrays d_pxq,
 * d_pyq (int32), d_pg1, d_pg2, d_pw (float) and d_pzbin (uint8; required when n_z > 1, else may be
 * NULL), each with room for n_z * npy * npx entries; *h_count receives the number of non-empty
 * pixels (the call synchronises the context's stream for it). The catalog d_xq..d_w, d_zbin is
 * the caller's device SoA as in mp3pcf_accumulate_moments. The sums are taken in FP64 (exact for
 * the products and their sums, so independent of the order of the additions). The pixel catalog
 * is an ordinary catalog for mp3pcf_accumulate_moments and the rest of the path: its moments are
 * the grid moments G_n^Delta, W_n^Delta and its contraction is Eq. UpsilonmuGrid (the outer sum
 * over pixels). Returns EINVAL for bad arguments (pixel_q < 1,
 * npx or npy < 1, more than 2^31 - 1 pixels, NULL pointers), ENOMEM if the context's scratch
 * cannot grow. */
mp3pcf_status mp3pcf_grid_catalog(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq, const int32_t* d_yq,
                                  const float* d_g1, const float* d_g2, const float* d_w, const uint8_t* d_zbin,
                                  const int64_t* h_origin, int64_t pixel_q, int32_t npx, int32_t npy,
                                  int32_t* d_pxq, int32_t* d_pyq, float* d_pg1, float* d_pg2, float* d_pw,
                                  uint8_t* d_pzbin, int64_t* h_count);

/* ---- Combined estimator (Sec. 3.3, Eq. CombinedEstimatorRegridding): the moments of the small
 * radial bins from the galaxies and those of the large bins from pixel catalogs (the grid-based
 * approximation above) of one or several resolutions. Level l (0 <= l < n_levels) covers bins
 * [h_b_start[l], h_b_start[l + 1]) (the last level up to n_bins) with pixels of h_pixel_q[l]
 * quanta on a grid whose origin is the lower corner of the catalog's extent (its bounding box,
 * or the fixed extent of mp3pcf_set_extent); bins [0, h_b_start[0]) are the discrete moments of
 * mp3pcf_accumulate_moments. For a centre galaxy i in pixel p_i of level l, its moments in the
 * level's bins are the pixel catalog's moments about the centre of p_i (G_n^Delta(p_i), as they
 * are: no division by the number of galaxies in the pixel); a galaxy whose pixel has no weight
 * gets zeros there. mp3pcf_contract_multipoles then gives the paper's combined estimate: both
 * bins discrete, Eq. CombinedEstimatorRegridding for one discrete and one grid bin, and
 * Eq. UpsilonmuGrid (the pixels' own contraction) for two grid bins of one level. Arguments as in
 * mp3pcf_accumulate_moments, plus n_levels >= 1, h_b_start (host, strictly increasing within
 * [0, n_bins)) and h_pixel_q (host, pixel sides >= 1). The pair count of mp3pcf_counts adds the
 * pixel pairs. Synchronises the stream once per level. EINVAL for bad levels or a grid of more
 * than 2^31 - 1 pixels, EUNSUPPORTED with cfg.exclude_degenerate; after this call
 * mp3pcf_moments_adjoint returns EUNSUPPORTED. */
mp3pcf_status mp3pcf_accumulate_moments_combined(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq,
                                                 const int32_t* d_yq, const float* d_g1, const float* d_g2,
                                                 const float* d_w, const uint8_t* d_zbin,
                                                 const uint8_t* d_centre_mask, int32_t n_levels,
                                                 const int32_t* h_b_start, const int64_t* h_pixel_q);

/* ---- Direct estimator of the third-order aperture mass (Sec. 5.3, Eq. MapDirectEstimator), an
 * estimate of <M_ap^3> independent of the 3PCF route, for unmasked catalogs. For every aperture
 * centre t (d_centres [n_centres][2] double, arcmin, in the frame of the fixed-point positions:
 * x = xq * quantum) and every radii triple a (d_theta_ap [n_ap][3] double, arcmin, > 0), writes
 * d_out[t][a][0] = sum over distinct galaxies i, j, k of w_i w_j w_k Q_1(r_i) Q_2(r_j) Q_3(r_k)
 * gt_i gt_j gt_k and d_out[t][a][1] = the same sum without the tangential shears gt (about the
 * centre), Q the filter of Eq. CrittendenQ; the estimate at the centre is their ratio and
 * <M_ap^3> is its average over apertures. Galaxies farther than rcut_factor * max(theta) from a
 * centre are left out (the paper uses 4). The catalog is the caller's device SoA (as in
 * mp3pcf_accumulate_moments, unsorted; zbin is not used); quantum comes from the context's
 * configuration. Sums in FP64 in the order of a fixed block reduction. Stream-ordered on the
 * context's stream. Returns EINVAL for bad arguments (negative counts, NULL pointers with
 * non-zero counts, rcut_factor <= 0, more than 2^31 - 1 apertures x triples). */
mp3pcf_status mp3pcf_map3_direct(mp3pcf_ctx* ctx, int64_t n, const int32_t* d_xq, const int32_t* d_yq,
                                 const float* d_g1, const float* d_g2, const float* d_w, int64_t n_centres,
                                 const double* d_centres, int64_t n_ap, const double* d_theta_ap,
                                 double rcut_factor, double* d_out);

/* ---- Failure injection, for tests of failure detection (host side only; nothing faults or
 * traps the GPU). MP3PCF_INJECT_WAIT_TIMEOUT: the tensor-core contraction issues no TMA copies,
 * so its bounded mbarrier waits (about a second each) run out; every role aborts, frees its
 * tensor memory and returns, the partial sums are zero, and the next mp3pcf_counts returns
 * ETIMEOUT; the context stays usable. MP3PCF_INJECT_ALLOC_FAILURE: mp3pcf_accumulate_moments
 * fails with ENOMEM before touching the workspace. on = 0 switches an injection off. */
enum { MP3PCF_INJECT_WAIT_TIMEOUT = 1, MP3PCF_INJECT_ALLOC_FAILURE = 2 };
mp3pcf_status mp3pcf_inject(mp3pcf_ctx* ctx, int32_t what, int32_t on);

/* ---- Batching form: many catalogs (mock realisations, each possibly tomographic), uneven
 * galaxy counts, through the whole path with captured CUDA graphs. */

/* One catalog in device memory (caller-owned, the layout of mp3pcf_accumulate_moments; zbin may
 * be NULL only when n_z = 1). */
typedef struct {
    int64_t n;
    const int32_t* xq;
    const int32_t* yq;
    const float* g1;
    const float* g2;
    const float* w;
    const uint8_t* zbin;
} mp3pcf_catalog_view;

/* Fixed patch extent h_extent[4] = (x0, y0, x1, y1) in position quanta (host), or NULL to go back
 * to measuring each catalog's extent. With a fixed extent mp3pcf_accumulate_moments makes no host
 * round trip for the cell grid; positions outside the extent (or zbin >= n_z) set an error that
 * mp3pcf_counts reports as EINVAL. Without a centre mask the whole path (accumulate, contract,
 * edge_correct with h_n_singular = NULL, to_gamma, to_map3) then runs without host
 * synchronisation and can be captured into a CUDA graph once the workspace has reached its size. */
mp3pcf_status mp3pcf_set_extent(mp3pcf_ctx* ctx, const int64_t* h_extent);

/* Runs the whole path (all centres, FP64 edge correction, centroid projection, aperture measures)
 * for n_cats catalogs inside the extent h_extent[4] and writes d_m8 [n_cats][n_z^3][n_ap][8]
 * (device) for the apertures d_theta_ap [n_ap][3]. The largest catalog runs first and sizes the
 * workspace; with use_graphs != 0 every other catalog's launches are captured into a CUDA graph
 * and replayed, one instantiated graph being updated in place (uneven counts only change kernel
 * parameters and grid sizes). Synchronises once at the end; EINVAL if a galaxy lies outside the
 * extent. The context's fixed extent and tracing switch are restored afterwards. */
mp3pcf_status mp3pcf_run_batch(mp3pcf_ctx* ctx, const mp3pcf_catalog_view* h_cats, int64_t n_cats,
                               const int64_t* h_extent, int64_t n_ap, const double* d_theta_ap, double* d_m8,
                               int32_t use_graphs);

/* CUDA-graph launches and instantiations made by mp3pcf_run_batch so far (host outputs). */
mp3pcf_status mp3pcf_graph_stats(mp3pcf_ctx* ctx, int64_t* h_launches, int64_t* h_instantiations);

/* ---- Adjoints (reverse mode), the differentiation form: dL/d(gamma_1, gamma_2, w) for a real
 * loss L of the aperture measures, by the chain to_map3 -> to_gamma -> edge_correct ->
 * contract_multipoles -> accumulate_moments taken backwards. For every complex quantity z the
 * gradient is grad z = dL/dRe z + i dL/dIm z (interleaved complex double, like the forward
 * buffers). All are stream-ordered and allocation happens only in the context's workspace. */

/* dL/dGamma^cen [n_z^3][4][n_bins][n_bins][n_phi] (OVERWRITTEN) of the aperture integral and
 * 8-measure combination (Sec. 5.2, App. C, Eqs. MapTrafo8_1-8) for apertures d_theta_ap
 * [n_ap][3], from d_grad_corr [n_z^3][n_ap][4] complex and/or d_grad_m8 [n_z^3][n_ap][8]
 * (either may be NULL; both NULL gives zeros). */
mp3pcf_status mp3pcf_to_map3_adjoint(mp3pcf_ctx* ctx, int64_t n_ap, const double* d_theta_ap,
                                     const double* d_grad_corr, const double* d_grad_m8,
                                     double* d_grad_gamma_cen);

/* dL/dGamma_n [n_z^3][4][2 n_max+1][n_bins][n_bins] (OVERWRITTEN) from
 * d_grad_gamma_phi [n_z^3][4][n_bins][n_bins][n_phi] of mp3pcf_to_gamma with the same projection
 * (the multipole sum and, for projection 1, the centroid factors). */
mp3pcf_status mp3pcf_to_gamma_adjoint(mp3pcf_ctx* ctx, int32_t projection, const double* d_grad_gamma_phi,
                                      double* d_grad_gamma_n);

/* dL/dUpsilon [n_z^3][4][n_max+1][n_bins][n_bins] and dL/dN [n_z^3][2 n_max+1][n_bins][n_bins]
 * (both OVERWRITTEN) of the edge-correction solve (Eqs. ModeCoupling, GammaMultipolesWithEC):
 * per system Y = A^{-H} dL/dGamma, dL/dA = -Y Gamma^H folded along the Toeplitz diagonals and
 * through the App. A symmetries. d_norm and d_gamma_n are the forward N and its solution; systems
 * that were singular contribute zeros. */
mp3pcf_status mp3pcf_edge_correct_adjoint(mp3pcf_ctx* ctx, const double* d_norm, const double* d_gamma_n,
                                          const double* d_grad_gamma_n, double* d_grad_upsilon,
                                          double* d_grad_norm);

/* Adjoint of mp3pcf_contract_multipoles and mp3pcf_accumulate_moments for the catalog of the
 * LAST accumulate call (the context still holds its sorted copy and moments): ADDS dL/dgamma_1,
 * dL/dgamma_2 and dL/dw per galaxy, in the caller's order, to d_grad_g1, d_grad_g2, d_grad_w
 * (float [n]; any may be NULL) given dL/dUpsilon and dL/dN. n and d_g1, d_g2, d_w must be the
 * catalog of that call (EINVAL if n differs). With exclude_degenerate the gradient of the
 * removed j = k terms is included. Arithmetic in the forward moment precision; the scatter to
 * neighbours uses atomics, so the result is not bit-reproducible. */
mp3pcf_status mp3pcf_moments_adjoint(mp3pcf_ctx* ctx, const double* d_grad_upsilon, const double* d_grad_norm,
                                     int64_t n, const float* d_g1, const float* d_g2, const float* d_w,
                                     float* d_grad_g1, float* d_grad_g2, float* d_grad_w);

/* Tracing. With timing on, every stage call records a pair of CUDA events on the context
 * stream around its kernels. mp3pcf_stage_times returns, per stage, the accumulated device time
 * in ms (h_ms[6], may be NULL) and the number of kernel launches (h_launches[6], may be NULL;
 * counted whether or not timing is on) since the last reset. Stages: 0 cell sort (step a0),
 * 1 moments (a1), 2 contraction (b1), 3 edge correction (c1), 4 to_gamma (c2), 5 to_map3 (c3).
 * reset != 0 clears the counters after reading. Synchronises the stream. */
mp3pcf_status mp3pcf_set_timing(mp3pcf_ctx* ctx, int32_t on);
mp3pcf_status mp3pcf_stage_times(mp3pcf_ctx* ctx, double* h_ms, int64_t* h_launches, int32_t reset);

/* Measurement service for rooflines (the paper has no counterpart). Runs, on the current device
 * and `stream`, a probe that keeps every SM busy with independent chains of one arithmetic
 * instruction: kind 0 FP32 FMA, 1 packed two-lane FP32 FMA (sm_100 and later), 2 FP64 FMA; or
 * with back-to-back tensor-core MMAs (tcgen05, M 128, N 256, FP32 accumulation in tensor
 * memory): kind 3 BF16 inputs, 4 TF32 inputs (ETIMEOUT if their bounded completion wait gave up).
 * Returns the best of three timed launches (after one warm-up) in *h_flops_per_s (2 flops per
 * FMA) and the SM clock during the probe in *h_sm_mhz (may be NULL). Allocates and frees two
 * small device buffers and synchronises the stream. EINVAL for another kind. */
mp3pcf_status mp3pcf_measure_peak(int32_t kind, void* stream, double* h_flops_per_s, double* h_sm_mhz);

/* Allocation-free form of mp3pcf_to_map3 (the paper has no counterpart: it is a service of this
 * library). For callers that may not allocate device memory, e.g. a plugin inside a host
 * application that owns all device memory through its own pool, or a service held to a fixed
 * memory budget: no context is needed and nothing is allocated. Same inputs and outputs as
 * mp3pcf_to_map3 (cfg as for mp3pcf_create; d_gamma_cen from mp3pcf_to_gamma with projection 1),
 * enqueued on `stream` (cudaStream_t, NULL: legacy default stream).
 * Scratch: one static 1 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits. It limits n_z^3 * n_ap to at most 255; larger requests
 * return EINVAL and enqueue nothing. Every call shares that array: calls whose work overlaps on
 * the GPU (two streams, or two host threads on one device) race and must be ordered by the
 * caller. The array's device address is looked up (cudaGetSymbolAddress) by every call made
 * outside stream capture and cached per CUDA context; a call made while `stream` is capturing
 * uses the cached address of the current context, so make a first call in that context outside
 * capture (again after cudaDeviceReset, which reloads the library's module), or the call
 * returns ECUDA. Either output may be NULL, not both.
 * Returns EINVAL for a bad configuration or argument, ECUDA if a CUDA call fails. */
mp3pcf_status mp3pcf_to_map3_noalloc(const mp3pcf_config* cfg, void* stream,
                                     const double* d_gamma_cen, int64_t n_ap,
                                     const double* d_theta_ap, double* d_corr, double* d_m8);

#ifdef __cplusplus
}
#endif

#endif /* MP3PCF_H */
