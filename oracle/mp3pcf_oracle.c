/*
 * FP64 CPU oracle for the multipole estimator of the shear three-point correlation function
 * (Porth, Heydenreich, Linke, Burger, Schneider 2023, "Efficient estimation of third-order shear
 * correlation functions").
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain reference that the CUDA library is checked
 * against. Only the tests, the smoke check and the benchmark's CPU-baseline / reference arm load
 * it. It shares no code with the CUDA library: it has its own configuration struct, its own
 * bin-edge table, its own neighbour search and its own arithmetic, all written from the paper.
 *
 * Conventions (readings of the paper where it is silent):
 *  - shear gamma_c = gamma_1 + i gamma_2; projected shear gamma(X; zeta) = -gamma_c e^{-2 i zeta}
 *    (Sec. 2.1, Eq. gammatx_def);
 *  - moments use e^{+i n phi} exactly as Eq. Gn_disc;
 *  - a pair (i,k) is in radial bin b iff e_b <= theta_ik < e_{b+1} (half-open), decided exactly
 *    on integer squared separations: r2 >= E2_b with E2_b = ceil((e_b/quantum)^2);
 *    e_b = theta_min * pow(theta_max/theta_min, b/n_bins);
 *  - the Gamma multipole series carries no 1/(2 pi): Gamma(phi) = sum_n Gamma_n e^{i n phi}, the
 *    only normalisation under which Eq. ModeCoupling holds as printed;
 *  - normalisation multipoles N_n are kept up to |n| = 2 n_max so that the full mode-coupling
 *    matrix N_{l-n}, l,n in [-n_max, n_max], is available (Eq. GammaMultipolesWithEC);
 *  - radial quadrature node of bin b: arithmetic midpoint (e_b+e_{b+1})/2 (or geometric), width
 *    e_{b+1}-e_b; angular nodes phi_k = (k+1/2) 2 pi / n_phi, k = 0..n_phi-1 (Sec. 4, 100 bins).
 *
 * Array layouts (complex numbers as interleaved re,im doubles; Z-triplet index
 * zt = (Z1*n_z + Z2)*n_z + Z3, centre in Z1, first radial bin with Z2, second with Z3):
 *   G      [n_centres][n_z][n_bins][2 n_max + 3]   m = -n_max-3 .. n_max-1
 *   W      [n_centres][n_z][n_bins][2 n_max + 1]   m = 0 .. 2 n_max
 *   ups    [n_z^3][4][n_max + 1][n_bins][n_bins]   n = 0 .. n_max
 *   norm   [n_z^3][2 n_max + 1][n_bins][n_bins]    n = 0 .. 2 n_max
 *   gam_n  [n_z^3][4][2 n_max + 1][n_bins][n_bins] n = -n_max .. n_max
 *   gam_phi[n_z^3][4][n_bins][n_bins][n_phi]
 *   corr   [n_z^3][n_ap][4]   <M^3>, <M* M^2>, <M M* M>, <M^2 M*>
 *   m8     [n_z^3][n_ap][8]   Map^3, <Mx Map Map>, <Map Mx Map>, <Map Map Mx>,
 *                             <Map Mx Mx>, <Mx Map Mx>, <Mx Mx Map>, Mx^3
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int32_t n_bins;
    double theta_min, theta_max; /* arcmin */
    int32_t n_max;
    int32_t n_phi;
    int32_t n_z;
    double quantum; /* arcmin per fixed-point unit */
    int32_t norm_truncate; /* 1: N_m = 0 for |m| > n_max in the coupling matrix */
    int32_t radial_nodes;  /* 0: arithmetic midpoint, 1: geometric midpoint */
    int32_t exclude_degenerate; /* 1: triplets with j = k are left out of Upsilon and N */
} orc_cfg;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ESINGULAR = 5 };

static int cfg_ok(const orc_cfg* c)
{
    if (!c) return 0;
    if (c->n_bins <= 0 || c->n_max < 0 || c->n_z <= 0 || c->n_phi <= 0) return 0;
    if (!(c->theta_min > 0) || !(c->theta_max > c->theta_min) || !(c->quantum > 0)) return 0;
    return 1;
}

static inline int nz3(const orc_cfg* c) { return c->n_z * c->n_z * c->n_z; }

/* ---- radial bins (Sec. 2.4: bins Theta_i = [Theta_low, Theta_up]; half-open reading) ---- */

int orc_edges(const orc_cfg* c, double* e, int64_t* e2q)
{
    if (!cfg_ok(c)) return ORC_EINVAL;
    for (int b = 0; b <= c->n_bins; ++b) {
        double eb = c->theta_min * pow(c->theta_max / c->theta_min, (double)b / c->n_bins);
        double t = eb / c->quantum;
        if (e) e[b] = eb;
        if (e2q) e2q[b] = (int64_t)ceil(t * t);
    }
    return ORC_OK;
}

static int bin_of(int64_t r2, const int64_t* e2q, int nb)
{
    if (r2 < e2q[0] || r2 >= e2q[nb]) return -1;
    int b = 0;
    while (r2 >= e2q[b + 1]) ++b;
    return b;
}

static double radial_node(const orc_cfg* c, const double* e, int b)
{
    return c->radial_nodes ? sqrt(e[b] * e[b + 1]) : 0.5 * (e[b] + e[b + 1]);
}

/* ---- a plain cell list: cells of side >= theta_max, each centre visits its 3x3 block ---- */

typedef struct {
    int64_t x0, y0, side, ncx, ncy;
    int64_t* start; /* ncx*ncy + 1 */
    int64_t* idx;   /* n */
} grid_t;

static void grid_free(grid_t* g)
{
    free(g->start);
    free(g->idx);
}

static int grid_build(grid_t* g, int64_t n, const int32_t* xq, const int32_t* yq, int64_t side)
{
    memset(g, 0, sizeof(*g));
    int64_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i == 0 || xq[i] < x0) x0 = xq[i];
        if (i == 0 || yq[i] < y0) y0 = yq[i];
        if (i == 0 || xq[i] > x1) x1 = xq[i];
        if (i == 0 || yq[i] > y1) y1 = yq[i];
    }
    g->x0 = x0;
    g->y0 = y0;
    g->side = side;
    g->ncx = (x1 - x0) / side + 1;
    g->ncy = (y1 - y0) / side + 1;
    int64_t nc = g->ncx * g->ncy;
    g->start = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    g->idx = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!g->start || !g->idx || !fill) {
        free(fill);
        grid_free(g);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (xq[i] - x0) / side, cy = (yq[i] - y0) / side;
        g->start[cy * g->ncx + cx + 1]++;
    }
    for (int64_t k = 0; k < nc; ++k) g->start[k + 1] += g->start[k];
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (xq[i] - x0) / side, cy = (yq[i] - y0) / side;
        int64_t cell = cy * g->ncx + cx;
        g->idx[g->start[cell] + fill[cell]++] = i;
    }
    free(fill);
    return ORC_OK;
}

static int64_t grid_side(const int64_t* e2q, int nb)
{
    return (int64_t)ceil(sqrt((double)e2q[nb])) + 2;
}

/* ---- stage (a): harmonic moments, Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization ---- */

int orc_moments(const orc_cfg* c, int64_t n, const int32_t* xq, const int32_t* yq,
                const float* g1, const float* g2, const float* w, const uint8_t* zbin,
                int64_t n_centres, const int64_t* centres, double* G_out, double* W_out)
{
    if (!cfg_ok(c) || n < 0 || n_centres < 0) return ORC_EINVAL;
    const int nb = c->n_bins, nmax = c->n_max, nz = c->n_z;
    const int MG = 2 * nmax + 3, MW = 2 * nmax + 1;
    int64_t* e2q = (int64_t*)malloc(sizeof(int64_t) * (nb + 1));
    orc_edges(c, NULL, e2q);
    grid_t g;
    if (grid_build(&g, n, xq, yq, grid_side(e2q, nb)) != ORC_OK) {
        free(e2q);
        return ORC_ENOMEM;
    }
    cplx* G = (cplx*)G_out;
    cplx* W = (cplx*)W_out;
    memset(G, 0, sizeof(cplx) * (size_t)n_centres * nz * nb * MG);
    memset(W, 0, sizeof(cplx) * (size_t)n_centres * nz * nb * MW);

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ci = 0; ci < n_centres; ++ci) {
        const int64_t i = centres[ci];
        const int64_t cx = (xq[i] - g.x0) / g.side, cy = (yq[i] - g.y0) / g.side;
        for (int64_t yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= g.ncy) continue;
            for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
                if (xx < 0 || xx >= g.ncx) continue;
                const int64_t cell = yy * g.ncx + xx;
                for (int64_t p = g.start[cell]; p < g.start[cell + 1]; ++p) {
                    const int64_t k = g.idx[p];
                    const int64_t dx = (int64_t)xq[k] - xq[i], dy = (int64_t)yq[k] - yq[i];
                    const int b = bin_of(dx * dx + dy * dy, e2q, nb);
                    if (b < 0) continue;
                    const double phi = atan2((double)dy, (double)dx); /* polar angle of theta_ik */
                    const int zk = zbin ? zbin[k] : 0;
                    const double wk = (double)w[k];
                    const cplx vk = wk * ((double)g1[k] + I * (double)g2[k]); /* w_k gamma_c,k */
                    cplx* Gp = G + (((size_t)ci * nz + zk) * nb + b) * MG;
                    cplx* Wp = W + (((size_t)ci * nz + zk) * nb + b) * MW;
                    for (int m = -nmax - 3; m <= nmax - 1; ++m) {
                        const double a = m * phi;
                        Gp[m + nmax + 3] += vk * (cos(a) + I * sin(a));
                    }
                    for (int m = 0; m <= 2 * nmax; ++m) {
                        const double a = m * phi;
                        Wp[m] += wk * (cos(a) + I * sin(a));
                    }
                }
            }
        }
    }
    grid_free(&g);
    free(e2q);
    return ORC_OK;
}

/* number of ordered pairs (i,k), i in centres, with theta_min <= theta_ik < theta_max */
int orc_count_pairs(const orc_cfg* c, int64_t n, const int32_t* xq, const int32_t* yq,
                    int64_t n_centres, const int64_t* centres, int64_t* count)
{
    if (!cfg_ok(c) || n < 0 || n_centres < 0) return ORC_EINVAL;
    const int nb = c->n_bins;
    int64_t* e2q = (int64_t*)malloc(sizeof(int64_t) * (nb + 1));
    orc_edges(c, NULL, e2q);
    grid_t g;
    if (grid_build(&g, n, xq, yq, grid_side(e2q, nb)) != ORC_OK) {
        free(e2q);
        return ORC_ENOMEM;
    }
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t ci = 0; ci < n_centres; ++ci) {
        const int64_t i = centres[ci];
        const int64_t cx = (xq[i] - g.x0) / g.side, cy = (yq[i] - g.y0) / g.side;
        for (int64_t yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= g.ncy) continue;
            for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
                if (xx < 0 || xx >= g.ncx) continue;
                const int64_t cell = yy * g.ncx + xx;
                for (int64_t p = g.start[cell]; p < g.start[cell + 1]; ++p) {
                    const int64_t k = g.idx[p];
                    const int64_t dx = (int64_t)xq[k] - xq[i], dy = (int64_t)yq[k] - yq[i];
                    if (bin_of(dx * dx + dy * dy, e2q, nb) >= 0) total++;
                }
            }
        }
    }
    *count = total;
    grid_free(&g);
    free(e2q);
    return ORC_OK;
}

/* ---- stage (b): multipole components, Eqs. Upsilon0_Derivation, Upsilon1-3 and
 *      3PCF_Normalization, with the tomographic form of Eq. tomoGn. Results are ADDED. ---- */

int orc_contract(const orc_cfg* c, const float* g1, const float* g2, const float* w,
                 const uint8_t* zbin, int64_t n_centres, const int64_t* centres,
                 const double* G_in, const double* W_in, double* ups_out, double* norm_out)
{
    if (!cfg_ok(c) || n_centres < 0) return ORC_EINVAL;
    const int nb = c->n_bins, nmax = c->n_max, nz = c->n_z;
    const int MG = 2 * nmax + 3, MW = 2 * nmax + 1, NN = nmax + 1, NW = 2 * nmax + 1;
    const cplx* G = (const cplx*)G_in;
    const cplx* W = (const cplx*)W_in;
    cplx* ups = (cplx*)ups_out;
    cplx* norm = (cplx*)norm_out;
#define GAT(ci, z, b, m) G[((((size_t)(ci)) * nz + (z)) * nb + (b)) * MG + (m) + nmax + 3]
#define WAT(ci, z, b, m) W[((((size_t)(ci)) * nz + (z)) * nb + (b)) * MW + (m)]
    const int64_t rows = (int64_t)nz3(c) * 5 * NW * nb; /* generous row space, filtered below */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < rows; ++r) {
        int64_t t = r;
        const int b1 = (int)(t % nb);
        t /= nb;
        const int n = (int)(t % NW);
        t /= NW;
        const int mu = (int)(t % 5); /* 0..3: Upsilon_mu ; 4: normalisation N */
        t /= 5;
        const int zt = (int)t;
        const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
        if (mu < 4 && n >= NN) continue;
        for (int b2 = 0; b2 < nb; ++b2) {
            cplx acc = 0;
            for (int64_t ci = 0; ci < n_centres; ++ci) {
                const int64_t i = centres[ci];
                if ((zbin ? zbin[i] : 0) != z1) continue;
                const double wi = (double)w[i];
                const cplx vi = wi * ((double)g1[i] + I * (double)g2[i]);
                switch (mu) {
                case 0: /* Upsilon_0,n = - sum w gamma G_{n-3}(T1) G_{-n-3}(T2) */
                    acc -= vi * GAT(ci, z2, b1, n - 3) * GAT(ci, z3, b2, -n - 3);
                    break;
                case 1: /* Upsilon_1,n = - sum w gamma* G_{n-1}(T1) G_{-n-1}(T2) */
                    acc -= conj(vi) * GAT(ci, z2, b1, n - 1) * GAT(ci, z3, b2, -n - 1);
                    break;
                case 2: /* Upsilon_2,n = - sum w gamma (G_{-n-1}(T1))* G_{-n-3}(T2) */
                    acc -= vi * conj(GAT(ci, z2, b1, -n - 1)) * GAT(ci, z3, b2, -n - 3);
                    break;
                case 3: /* Upsilon_3,n = - sum w gamma G_{n-3}(T1) (G_{n-1}(T2))* */
                    acc -= vi * GAT(ci, z2, b1, n - 3) * conj(GAT(ci, z3, b2, n - 1));
                    break;
                default: /* N_n = sum w W_n(T1) (W_n(T2))* */
                    acc += wi * WAT(ci, z2, b1, n) * conj(WAT(ci, z3, b2, n));
                }
            }
            if (mu < 4)
                ups[((((size_t)zt * 4 + mu) * NN + n) * nb + b1) * nb + b2] += acc;
            else
                norm[(((size_t)zt * NW + n) * nb + b1) * nb + b2] += acc;
        }
    }
#undef GAT
#undef WAT
    return ORC_OK;
}

/* ---- edge correction: solve sum_n N_{l-n} Gamma_n = Upsilon_l, l,n in [-n_max, n_max]
 *      (Eqs. ModeCoupling, GammaMultipolesWithEC), negative orders from the symmetries of
 *      App. A (Upsilon_{0,-n}(i,j) = Upsilon_{0,n}(j,i), Upsilon_{2,-n}(i,j) =
 *      Upsilon_{3,n}(j,i), N_{-n}(i,j) = N_n(j,i), with Z2 <-> Z3). ---- */

/* Gaussian elimination with partial pivoting, in place; A is D x D row-major, B is D x R. */
/* With exclude_degenerate: subtracts from Upsilon and N (as produced by orc_contract) the
 * contributions of the triplets with j = k. In the sums of Eqs. Upsilon0_Derivation, Upsilon1-3
 * and 3PCF_Normalization such a triplet pairs a neighbour k with itself, so it only occurs for
 * b1 = b2 (and Z2 = Z3 = Z of k); each term is the product of the two moment terms of that one
 * neighbour, evaluated here straight from those products for every n. */
int orc_degenerate_correction(const orc_cfg* c, int64_t n, const int32_t* xq, const int32_t* yq,
                              const float* g1, const float* g2, const float* w, const uint8_t* zbin,
                              int64_t n_centres, const int64_t* centres, double* ups_io, double* norm_io)
{
    if (!cfg_ok(c) || n < 0 || n_centres < 0) return ORC_EINVAL;
    if (!c->exclude_degenerate) return ORC_OK;
    const int nb = c->n_bins, nmax = c->n_max, nz = c->n_z, NN = nmax + 1, NW = 2 * nmax + 1;
    int64_t* e2q = (int64_t*)malloc(sizeof(int64_t) * (nb + 1));
    orc_edges(c, NULL, e2q);
    cplx* ups = (cplx*)ups_io;
    cplx* norm = (cplx*)norm_io;
    for (int64_t ci = 0; ci < n_centres; ++ci) {
        const int64_t i = centres[ci];
        const int z1 = zbin ? zbin[i] : 0;
        const double wi = (double)w[i];
        const cplx vi = wi * ((double)g1[i] + I * (double)g2[i]);
        for (int64_t k = 0; k < n; ++k) {
            const int64_t dx = (int64_t)xq[k] - xq[i], dy = (int64_t)yq[k] - yq[i];
            const int b = bin_of(dx * dx + dy * dy, e2q, nb);
            if (b < 0) continue;
            const double phi = atan2((double)dy, (double)dx);
            const int zk = zbin ? zbin[k] : 0;
            const int zt = (z1 * nz + zk) * nz + zk;
            const double wk = (double)w[k];
            const cplx vk = wk * ((double)g1[k] + I * (double)g2[k]);
            for (int m = 0; m <= nmax; ++m) {
                /* the same neighbour as the X and the Y moment term of each component */
                const cplx x0 = vk * cexp(I * (m - 3) * phi), y0 = vk * cexp(I * (-m - 3) * phi);
                const cplx x1 = vk * cexp(I * (m - 1) * phi), y1 = vk * cexp(I * (-m - 1) * phi);
                const cplx x2 = conj(vk * cexp(I * (-m - 1) * phi)), y2 = vk * cexp(I * (-m - 3) * phi);
                const cplx x3 = vk * cexp(I * (m - 3) * phi), y3 = conj(vk * cexp(I * (m - 1) * phi));
                const size_t at = (size_t)b * nb + b;
                ups[(((size_t)zt * 4 + 0) * NN + m) * nb * nb + at] -= -vi * x0 * y0;
                ups[(((size_t)zt * 4 + 1) * NN + m) * nb * nb + at] -= -conj(vi) * x1 * y1;
                ups[(((size_t)zt * 4 + 2) * NN + m) * nb * nb + at] -= -vi * x2 * y2;
                ups[(((size_t)zt * 4 + 3) * NN + m) * nb * nb + at] -= -vi * x3 * y3;
            }
            for (int m = 0; m < NW; ++m) {
                const cplx wx = wk * cexp(I * m * phi);
                norm[((size_t)zt * NW + m) * nb * nb + (size_t)b * nb + b] -= wi * wx * conj(wx);
            }
        }
    }
    free(e2q);
    return ORC_OK;
}

static int solve_lu(int D, int R, cplx* A, cplx* B)
{
    for (int k = 0; k < D; ++k) {
        int piv = k;
        double best = cabs(A[k * D + k]);
        for (int r = k + 1; r < D; ++r) {
            double v = cabs(A[r * D + k]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 0)) return ORC_ESINGULAR;
        if (piv != k) {
            for (int j = 0; j < D; ++j) {
                cplx t = A[k * D + j];
                A[k * D + j] = A[piv * D + j];
                A[piv * D + j] = t;
            }
            for (int j = 0; j < R; ++j) {
                cplx t = B[k * R + j];
                B[k * R + j] = B[piv * R + j];
                B[piv * R + j] = t;
            }
        }
        for (int r = k + 1; r < D; ++r) {
            const cplx f = A[r * D + k] / A[k * D + k];
            if (f == 0) continue;
            for (int j = k; j < D; ++j) A[r * D + j] -= f * A[k * D + j];
            for (int j = 0; j < R; ++j) B[r * R + j] -= f * B[k * R + j];
        }
    }
    for (int k = D - 1; k >= 0; --k) {
        for (int j = 0; j < R; ++j) {
            cplx s = B[k * R + j];
            for (int q = k + 1; q < D; ++q) s -= A[k * D + q] * B[q * R + j];
            B[k * R + j] = s / A[k * D + k];
        }
    }
    return ORC_OK;
}

int orc_edge_correct(const orc_cfg* c, const double* ups_in, const double* norm_in,
                     double* gam_out, int64_t* n_singular)
{
    if (!cfg_ok(c)) return ORC_EINVAL;
    const int nb = c->n_bins, nmax = c->n_max, nz = c->n_z;
    const int NN = nmax + 1, NW = 2 * nmax + 1, D = 2 * nmax + 1;
    const cplx* ups = (const cplx*)ups_in;
    const cplx* norm = (const cplx*)norm_in;
    cplx* gam = (cplx*)gam_out;
    int64_t nsing = 0;
    const int64_t systems = (int64_t)nz3(c) * nb * nb;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nsing)
    for (int64_t s = 0; s < systems; ++s) {
        const int b2 = (int)(s % nb), b1 = (int)((s / nb) % nb);
        const int zt = (int)(s / ((int64_t)nb * nb));
        const int z1 = zt / (nz * nz), z2 = (zt / nz) % nz, z3 = zt % nz;
        const int zs = (z1 * nz + z3) * nz + z2; /* Z2 <-> Z3 swapped triplet */
        cplx* A = (cplx*)malloc(sizeof(cplx) * D * D);
        cplx* B = (cplx*)malloc(sizeof(cplx) * D * 4);
        /* N_m for m in [-2 n_max, 2 n_max] */
        for (int l = -nmax; l <= nmax; ++l) {
            for (int nn = -nmax; nn <= nmax; ++nn) {
                const int m = l - nn;
                cplx v;
                if (c->norm_truncate && (m > nmax || m < -nmax))
                    v = 0;
                else if (m >= 0)
                    v = norm[(((size_t)zt * NW + m) * nb + b1) * nb + b2];
                else
                    v = norm[(((size_t)zs * NW + (-m)) * nb + b2) * nb + b1];
                A[(l + nmax) * D + (nn + nmax)] = v;
            }
            for (int mu = 0; mu < 4; ++mu) {
                cplx v;
                if (l >= 0) {
                    v = ups[((((size_t)zt * 4 + mu) * NN + l) * nb + b1) * nb + b2];
                } else {
                    const int mus = (mu == 2) ? 3 : (mu == 3) ? 2 : mu;
                    v = ups[((((size_t)zs * 4 + mus) * NN + (-l)) * nb + b2) * nb + b1];
                }
                B[(l + nmax) * 4 + mu] = v;
            }
        }
        const cplx n0 = A[nmax * D + nmax];
        int st = (n0 == 0) ? ORC_ESINGULAR : solve_lu(D, 4, A, B);
        for (int nn = 0; nn < D; ++nn)
            for (int mu = 0; mu < 4; ++mu)
                gam[((((size_t)zt * 4 + mu) * D + nn) * nb + b1) * nb + b2] =
                    (st == ORC_OK) ? B[nn * 4 + mu] : (NAN + I * NAN);
        if (st != ORC_OK) nsing++;
        free(A);
        free(B);
    }
    if (n_singular) *n_singular = nsing;
    return nsing ? ORC_ESINGULAR : ORC_OK;
}

/* ---- multipoles -> Gamma^x(phi) -> Gamma^cen (Sec. 2.3, Eqs. X2Centroid0-3 with the
 *      phi_1-free rotation factors printed below them) ---- */

/* factor turning Gamma^x_mu(t1, t2, phi) into Gamma^cen_mu */
static cplx cen_factor(int mu, double t1, double t2, double phi)
{
    const cplx ep = cexp(I * phi), em = cexp(-I * phi);
    const cplx R1 = (t1 + t2 * em) / (t1 + t2 * ep);
    const cplx R2 = (t2 * em - 2 * t1) / (t2 * ep - 2 * t1);
    const cplx R3 = (t1 - 2 * t2 * em) / (t1 - 2 * t2 * ep);
    switch (mu) {
    case 0: return R1 * R2 * R3 * cexp(3 * I * phi);
    case 1: return R2 * R3 / R1 * cexp(I * phi);
    case 2: return R1 * R3 / R2 * cexp(3 * I * phi);
    default: return R1 * R2 / R3 * cexp(-I * phi);
    }
}

int orc_cen_factor(int mu, double t1, double t2, double phi, double* out)
{
    cplx f = cen_factor(mu, t1, t2, phi);
    out[0] = creal(f);
    out[1] = cimag(f);
    return ORC_OK;
}

/* projection 0: x-projection at phi_k; 1: centroid projection at phi_k; 2: x-projection averaged
 * over the angular bin around phi_k (Sec. 2.4, the binned 3PCF) */
int orc_to_gamma(const orc_cfg* c, const double* gam_in, int32_t projection, double* out)
{
    if (!cfg_ok(c) || projection < 0 || projection > 2) return ORC_EINVAL;
    const int nb = c->n_bins, nmax = c->n_max, D = 2 * nmax + 1, np = c->n_phi;
    double* e = (double*)malloc(sizeof(double) * (nb + 1));
    orc_edges(c, e, NULL);
    const cplx* gam = (const cplx*)gam_in;
    cplx* gp = (cplx*)out;
    const int64_t rows = (int64_t)nz3(c) * 4 * nb * nb;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        const int b2 = (int)(r % nb), b1 = (int)((r / nb) % nb);
        const int64_t zm = r / ((int64_t)nb * nb); /* zt*4 + mu */
        const int mu = (int)(zm % 4);
        for (int k = 0; k < np; ++k) {
            const double phi = (k + 0.5) * 2.0 * M_PI / np;
            cplx s = 0;
            for (int nn = -nmax; nn <= nmax; ++nn) {
                const cplx gn = gam[((size_t)zm * D + (nn + nmax)) * nb * nb + (size_t)b1 * nb + b2];
                /* projection 2: mean of e^{i n phi} over [phi - h, phi + h), h = pi / np */
                const double h = M_PI / np;
                const double avg = (projection == 2 && nn != 0) ? sin(nn * h) / (nn * h) : 1.0;
                s += gn * avg * (cos(nn * phi) + I * sin(nn * phi));
            }
            if (projection == 1) s *= cen_factor(mu, radial_node(c, e, b1), radial_node(c, e, b2), phi);
            gp[(((size_t)zm * nb + b1) * nb + b2) * np + k] = s;
        }
    }
    free(e);
    return ORC_OK;
}

/* ---- third-order aperture measures (Sec. 5.2, Eqs. MFrom3pcfTheory(b); filters of App. C
 *      Eq. 3pcftomap3_helpers and the F_0, F_1 expressions, the other two by cyclic label
 *      permutations of F_1; 8-equation combination Eqs. MapTrafo8_1-8) ---- */

/* q-vectors of Eq. QvecDef in the frame where theta_1-vector lies on the real axis */
static void qvecs(double t1, double t2, double phi, cplx q[3])
{
    const cplx v1 = t1, v2 = t2 * cexp(I * phi);
    q[0] = -(v1 + v2) / 3.0;
    q[1] = (2.0 * v1 - v2) / 3.0;
    q[2] = (2.0 * v2 - v1) / 3.0;
}

/* the printed F_1 expression with vertex labels rotated by s: slot a of the printed formula
 * takes vertex (a + s) mod 3, i.e. s = 1 is the permutation (231) and s = 2 is (312) */
static cplx filter_F1_rot(int s, double t1, double t2, double phi, const double th[3])
{
    cplx q[3];
    qvecs(t1, t2, phi, q);
    const double T4 = (th[0] * th[0] * th[1] * th[1] + th[0] * th[0] * th[2] * th[2] +
                       th[1] * th[1] * th[2] * th[2]) / 3.0;
    const double T2 = sqrt(T4), T6 = T2 * T4;
    const double S = th[0] * th[0] * th[1] * th[1] * th[2] * th[2] / T6;
    const double M = S * t1 * t2 / (2.0 * M_PI * T4);
    double Z = 0;
    for (int i = 0; i < 3; ++i) {
        const double a = th[i] * th[i], b = th[(i + 1) % 3] * th[(i + 1) % 3],
                     cc = th[(i + 2) % 3] * th[(i + 2) % 3];
        Z += (-a + 2 * b + 2 * cc) * creal(q[i] * conj(q[i]));
    }
    Z /= 6.0 * T4;
    cplx f[3], g[3];
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        const double a = th[i] * th[i], b = th[i1] * th[i1], cc = th[i2] * th[i2];
        const cplx r = conj(q[i]) * (q[i1] - q[i2]) / creal(q[i] * conj(q[i]));
        f[i] = (b + cc) / (2 * T2) + r * (b - cc) / (6 * T2);
        g[i] = b * cc / T4 + r * a * (cc - b) / (3 * T4);
    }
    /* rotated labels: slot 1 -> index s, slot 2 -> s+1, slot 3 -> s+2 */
    const int i1 = s % 3, i2 = (s + 1) % 3, i3 = (s + 2) % 3;
    const double th1 = th[i1], th3 = th[i3];
    const cplx q1 = q[i1], q2 = q[i2], q3 = q[i3];
    const cplx f1 = f[i1], f2 = f[i2], f3 = f[i3], gg2 = g[i2];
    const double aq = creal(q[0] * conj(q[0])) * creal(q[1] * conj(q[1])) * creal(q[2] * conj(q[2]));
    const double q2sq = creal(q2 * conj(q2));
    const cplx q2c = conj(q2);
    cplx term = aq / (24 * T6) * conj(f3) * conj(f3) * conj(f1) * conj(f1) * f2 * f2;
    term -= (1.0 / 9.0) * q3 * q1 * q2c * q2c / T4 * conj(f3) * conj(f1) * f2 * conj(gg2);
    term += (1.0 / 27.0) * (q3 * q3 * q1 * q1 * q2c * q2c * q2c * q2c / (aq * T2) * conj(gg2) * conj(gg2) +
                            2 * th3 * th3 * th1 * th1 / T4 * q3 * q1 * q2c * q2c / (q2sq * T2) *
                                conj(f3) * conj(f1));
    return M * exp(-Z) * term;
}

static cplx filter_F0(double t1, double t2, double phi, const double th[3])
{
    cplx q[3];
    qvecs(t1, t2, phi, q);
    const double T4 = (th[0] * th[0] * th[1] * th[1] + th[0] * th[0] * th[2] * th[2] +
                       th[1] * th[1] * th[2] * th[2]) / 3.0;
    const double T2 = sqrt(T4), T6 = T2 * T4;
    const double S = th[0] * th[0] * th[1] * th[1] * th[2] * th[2] / T6;
    const double M = S * t1 * t2 / (2.0 * M_PI * T4);
    double Z = 0;
    cplx prod = 1;
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        const double a = th[i] * th[i], b = th[i1] * th[i1], cc = th[i2] * th[i2];
        Z += (-a + 2 * b + 2 * cc) * creal(q[i] * conj(q[i]));
        const cplx r = conj(q[i]) * (q[i1] - q[i2]) / creal(q[i] * conj(q[i]));
        const cplx fi = (b + cc) / (2 * T2) + r * (b - cc) / (6 * T2);
        prod *= conj(fi) * conj(fi);
    }
    Z /= 6.0 * T4;
    const double aq = creal(q[0] * conj(q[0])) * creal(q[1] * conj(q[1])) * creal(q[2] * conj(q[2]));
    return M / 24.0 * aq / T6 * prod * exp(-Z);
}

/* F_mu(t1, t2, phi; theta_1..3). mu = 0: F_0. For mu = 1..3 the correlator has its conjugate
 * at vertex mu. The F_1 printed in App. C, read with the q-vectors of Eq. QvecDef, is the kernel
 * whose conjugate sits at vertex 2 (this follows from writing <M* M M> etc. out from
 * Eqs. MapGamma and CrittendenQ and the centroid projection, and is checked by direct
 * integration in the tests). So the printed expression is rotated until its special vertex
 * lands on vertex mu: mu = 1 -> rotation 2, mu = 2 -> rotation 0, mu = 3 -> rotation 1. */
static cplx filter_F(int mu, double t1, double t2, double phi, const double th[3])
{
    return mu == 0 ? filter_F0(t1, t2, phi, th) : filter_F1_rot((mu + 1) % 3, t1, t2, phi, th);
}

int orc_filter(int32_t mu, double t1, double t2, double phi, const double* th, double* out)
{
    if (mu < 0 || mu > 3) return ORC_EINVAL;
    cplx f = filter_F(mu, t1, t2, phi, th);
    out[0] = creal(f);
    out[1] = cimag(f);
    return ORC_OK;
}

/* the real measures from the four complex correlators, Eqs. MapTrafo8_1-8 */
static void combine8(const cplx cc[4], double m8[8])
{
    const cplx c0 = cc[0], c1 = cc[1], c2 = cc[2], c3 = cc[3];
    m8[0] = creal(c3 + c2 + c1 + c0) / 4;
    m8[1] = cimag(c3 + c2 - c1 + c0) / 4;
    m8[2] = cimag(c3 - c2 + c1 + c0) / 4;
    m8[3] = cimag(-c3 + c2 + c1 + c0) / 4;
    m8[4] = creal(c3 + c2 - c1 - c0) / 4;
    m8[5] = creal(c3 - c2 + c1 - c0) / 4;
    m8[6] = creal(-c3 + c2 + c1 - c0) / 4;
    m8[7] = cimag(c3 + c2 + c1 - c0) / 4;
}

int orc_combine8(const double* corr, double* m8)
{
    cplx cc[4];
    for (int mu = 0; mu < 4; ++mu) cc[mu] = corr[2 * mu] + I * corr[2 * mu + 1];
    combine8(cc, m8);
    return ORC_OK;
}

int orc_to_map3(const orc_cfg* c, const double* gcen_in, int64_t n_ap, const double* theta_ap,
                double* corr_out, double* m8_out)
{
    if (!cfg_ok(c) || n_ap < 0) return ORC_EINVAL;
    const int nb = c->n_bins, np = c->n_phi;
    double* e = (double*)malloc(sizeof(double) * (nb + 1));
    orc_edges(c, e, NULL);
    const cplx* gc = (const cplx*)gcen_in;
    cplx* corr = (cplx*)corr_out;
    const double dphi = 2.0 * M_PI / np;
    const int64_t jobs = (int64_t)nz3(c) * n_ap;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t jb = 0; jb < jobs; ++jb) {
        const int64_t zt = jb / n_ap, a = jb % n_ap;
        const double* th = theta_ap + 3 * a;
        cplx cc[4] = {0, 0, 0, 0};
        for (int mu = 0; mu < 4; ++mu) {
            for (int b1 = 0; b1 < nb; ++b1) {
                const double t1 = radial_node(c, e, b1), d1 = e[b1 + 1] - e[b1];
                for (int b2 = 0; b2 < nb; ++b2) {
                    const double t2 = radial_node(c, e, b2), d2 = e[b2 + 1] - e[b2];
                    for (int k = 0; k < np; ++k) {
                        const double phi = (k + 0.5) * dphi;
                        const cplx gv = gc[((((size_t)zt * 4 + mu) * nb + b1) * nb + b2) * np + k];
                        cc[mu] += gv * filter_F(mu, t1, t2, phi, th) * d1 * d2 * dphi;
                    }
                }
            }
        }
        for (int mu = 0; mu < 4; ++mu) corr[(size_t)jb * 4 + mu] = cc[mu];
        combine8(cc, m8_out + (size_t)jb * 8);
    }
    free(e);
    return ORC_OK;
}

/* ---- the shorter four-equation form of the aperture measures (App. C, Eqs. MapTrafo4_1-4):
 *        Map^3          = Re[A123 + A132 + A231 + M3] / 4
 *        <Map^2 Mx>     = Im[-A123 + A132 + A231 + M3] / 4
 *        <Map Mx^2>     = Re[A123 + A132 - A231 - M3] / 4
 *        <Mx^3>         = Im[A123 + A132 + A231 - M3] / 4
 *      with M3 = <M^3>(t1, t2, t3) and Aabc the correlator with one conjugated factor at the radii
 *      (ta, tb, tc). As printed, the equations place the conjugate on the LAST radius of each list
 *      (<M^2 M^*>, the convention of the paper's reference for these forms): with the conjugate
 *      first, as <M^* M^2> is defined in Eq. MFrom3pcfTheory, A123 and A132 would be the same
 *      number and no term would conjugate t3, and the four measures would not be recovered. So
 *      Aabc = <M^* M^2>(tc, ta, tb): the Gamma_1 / F_1 correlator at (t3, t1, t2), (t2, t1, t3) and
 *      (t1, t2, t3). It equals the eight-equation form where the correlators obey the relabelling
 *      symmetries the appendix invokes, i.e. up to the quadrature and binning of the estimated
 *      3PCF. ---- */
int orc_combine4(const double* m3, const double* a123, const double* a132, const double* a231, double* m4)
{
    const cplx M3 = m3[0] + I * m3[1];
    const cplx A123 = a123[0] + I * a123[1], A132 = a132[0] + I * a132[1], A231 = a231[0] + I * a231[1];
    m4[0] = creal(A123 + A132 + A231 + M3) / 4.0;
    m4[1] = cimag(-A123 + A132 + A231 + M3) / 4.0;
    m4[2] = creal(A123 + A132 - A231 - M3) / 4.0;
    m4[3] = cimag(A123 + A132 + A231 - M3) / 4.0;
    return ORC_OK;
}

/* m4 [n_z^3][n_ap][4] = (Map^3, <Map^2 Mx>, <Map Mx^2>, <Mx^3>) at each radii triple */
int orc_to_map3_four(const orc_cfg* c, const double* gcen_in, int64_t n_ap, const double* theta_ap,
                     double* m4_out)
{
    if (!cfg_ok(c) || n_ap < 0) return ORC_EINVAL;
    const int64_t z3 = nz3(c), na = n_ap > 0 ? n_ap : 1;
    double* th3 = (double*)malloc(sizeof(double) * 9 * na);
    double* corr = (double*)malloc(sizeof(double) * 2 * 4 * z3 * 3 * na);
    double* m8 = (double*)malloc(sizeof(double) * 8 * z3 * 3 * na);
    for (int64_t a = 0; a < n_ap; ++a) {
        const double t1 = theta_ap[3 * a], t2 = theta_ap[3 * a + 1], t3 = theta_ap[3 * a + 2];
        const double order[3][3] = {{t3, t1, t2}, {t2, t1, t3}, {t1, t2, t3}};  /* A123, A132, A231 */
        for (int q = 0; q < 3; ++q)
            for (int i = 0; i < 3; ++i) th3[(3 * a + q) * 3 + i] = order[q][i];
    }
    int st = orc_to_map3(c, gcen_in, 3 * n_ap, th3, corr, m8);
    if (st == ORC_OK)
        for (int64_t zt = 0; zt < z3; ++zt)
            for (int64_t a = 0; a < n_ap; ++a) {
                const double* cc = corr + 2 * (zt * 3 * n_ap + 3 * a) * 4;  /* [ordering][mu] complex */
                orc_combine4(cc + 16, cc + 2, cc + 8 + 2, cc + 16 + 2, m4_out + (zt * n_ap + a) * 4);
            }
    free(th3);
    free(corr);
    free(m8);
    return st;
}

/* ---- brute-force triplet sums straight from the definitions (Sec. 2.2 Eqs. Gamma0_def -
 *      Gamma3_def in the x-projection Eq. xprojection; Eqs. TripletUpsilon and TripletNorm):
 *      for every ordered triplet (i, j, k) with theta_ij in bin b1 and theta_ik in bin b2
 *      (j = k included), phi = varphi_ik - varphi_ij,
 *        ups_n [mu][n][b1][b2]    += T_mu e^{-i n phi}            (n = 0..n_max)
 *        norm_n[n][b1][b2]        += w_i w_j w_k e^{-i n phi}     (n = 0..2 n_max)
 *        ups_b [mu][b1][b2][kphi] += T_mu   with phi binned into n_phib bins of [0, 2 pi)
 *        norm_b[b1][b2][kphi]     += w_i w_j w_k
 *        upsc_b[mu][b1][b2][kphi] += T^cen_mu (centroid projection, Eqs. centroidprojection,
 *                                    QvecDef)
 *      T_mu = w_i w_j w_k * product of projected shears gamma(X_a; zeta_a), conjugated at
 *      vertex mu for mu >= 1. The largest |T^cen - T^x * factor| / max|T^x| over all triplets
 *      (the per-triplet x -> centroid identity) is returned in *p5_dev. Outputs are overwritten.
 *      Tomographic index as in the header. ---- */

static inline cplx proj(cplx gc, double zeta, int conjugate)
{
    const cplx g = -gc * cexp(-2.0 * I * zeta); /* Eq. gammatx_def */
    return conjugate ? conj(g) : g;
}

static inline cplx proj_cen(cplx gc, cplx q, int conjugate)
{
    const cplx g = -gc * conj(q) / q; /* e^{-2 i zeta} = conj(q)/q, Eq. centroidprojection */
    return conjugate ? conj(g) : g;
}

int orc_brute(const orc_cfg* c, int64_t n, const int32_t* xq, const int32_t* yq,
              const float* g1, const float* g2, const float* w, const uint8_t* zbin,
              int32_t n_phib, double* ups_n_out, double* norm_n_out, double* ups_b_out,
              double* norm_b_out, double* upsc_b_out, double* p5_dev)
{
    if (!cfg_ok(c) || n < 0 || n_phib <= 0) return ORC_EINVAL;
    const int nb = c->n_bins, nmax = c->n_max, nz = c->n_z, NN = nmax + 1, NW = 2 * nmax + 1;
    const int Z3 = nz3(c);
    const size_t s_un = (size_t)Z3 * 4 * NN * nb * nb, s_nn = (size_t)Z3 * NW * nb * nb;
    const size_t s_ub = (size_t)Z3 * 4 * nb * nb * n_phib, s_nb = (size_t)Z3 * nb * nb * n_phib;
    int64_t* e2q = (int64_t*)malloc(sizeof(int64_t) * (nb + 1));
    orc_edges(c, NULL, e2q);
    cplx* ups_n = (cplx*)ups_n_out;
    cplx* norm_n = (cplx*)norm_n_out;
    cplx* ups_b = (cplx*)ups_b_out;
    cplx* norm_b = (cplx*)norm_b_out;
    cplx* upsc_b = (cplx*)upsc_b_out;
    memset(ups_n, 0, s_un * sizeof(cplx));
    memset(norm_n, 0, s_nn * sizeof(cplx));
    memset(ups_b, 0, s_ub * sizeof(cplx));
    memset(norm_b, 0, s_nb * sizeof(cplx));
    memset(upsc_b, 0, s_ub * sizeof(cplx));
    double dev = 0, tmax = 0;
#pragma omp parallel
    {
        cplx* lun = (cplx*)calloc(s_un, sizeof(cplx));
        cplx* lnn = (cplx*)calloc(s_nn, sizeof(cplx));
        cplx* lub = (cplx*)calloc(s_ub, sizeof(cplx));
        cplx* lnb = (cplx*)calloc(s_nb, sizeof(cplx));
        cplx* luc = (cplx*)calloc(s_ub, sizeof(cplx));
        int* nbr = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
        int* nbb = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
        double ldev = 0, ltmax = 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n; ++i) {
            int cnt = 0;
            for (int64_t k = 0; k < n; ++k) {
                const int64_t dx = (int64_t)xq[k] - xq[i], dy = (int64_t)yq[k] - yq[i];
                const int b = bin_of(dx * dx + dy * dy, e2q, nb);
                if (b >= 0) {
                    nbr[cnt] = (int)k;
                    nbb[cnt] = b;
                    cnt++;
                }
            }
            const int z1 = zbin ? zbin[i] : 0;
            const double wi = w[i];
            const cplx gi = (double)g1[i] + I * (double)g2[i];
            for (int a = 0; a < cnt; ++a) {
                const int j = nbr[a], b1 = nbb[a];
                const double dxj = (double)((int64_t)xq[j] - xq[i]), dyj = (double)((int64_t)yq[j] - yq[i]);
                const double phi1 = atan2(dyj, dxj);
                const int z2 = zbin ? zbin[j] : 0;
                const cplx gj = (double)g1[j] + I * (double)g2[j];
                for (int bb = 0; bb < cnt; ++bb) {
                    const int k = nbr[bb], b2 = nbb[bb];
                    if (c->exclude_degenerate && k == j) continue;
                    const double dxk = (double)((int64_t)xq[k] - xq[i]), dyk = (double)((int64_t)yq[k] - yq[i]);
                    const double phi2 = atan2(dyk, dxk);
                    const int z3 = zbin ? zbin[k] : 0;
                    const int zt = (z1 * nz + z2) * nz + z3;
                    const cplx gk = (double)g1[k] + I * (double)g2[k];
                    const double www = wi * (double)w[j] * (double)w[k];
                    const double phi = phi2 - phi1;
                    /* x-projection angles, Eq. xprojection */
                    const double z1a = 0.5 * (phi1 + phi2), z2a = phi1, z3a = phi2;
                    cplx T[4];
                    T[0] = www * proj(gi, z1a, 0) * proj(gj, z2a, 0) * proj(gk, z3a, 0);
                    T[1] = www * proj(gi, z1a, 1) * proj(gj, z2a, 0) * proj(gk, z3a, 0);
                    T[2] = www * proj(gi, z1a, 0) * proj(gj, z2a, 1) * proj(gk, z3a, 0);
                    T[3] = www * proj(gi, z1a, 0) * proj(gj, z2a, 0) * proj(gk, z3a, 1);
                    /* multipoles: e^{-i n phi} by recurrence */
                    const cplx step = cexp(-I * phi);
                    cplx e = 1;
                    for (int nn = 0; nn <= 2 * nmax; ++nn) {
                        if (nn <= nmax)
                            for (int mu = 0; mu < 4; ++mu)
                                lun[((((size_t)zt * 4 + mu) * NN + nn) * nb + b1) * nb + b2] += T[mu] * e;
                        lnn[(((size_t)zt * NW + nn) * nb + b1) * nb + b2] += www * e;
                        e *= step;
                    }
                    /* angular bin of phi in [0, 2 pi) */
                    double pm = fmod(phi, 2.0 * M_PI);
                    if (pm < 0) pm += 2.0 * M_PI;
                    int kb = (int)(pm / (2.0 * M_PI) * n_phib);
                    if (kb >= n_phib) kb = n_phib - 1;
                    for (int mu = 0; mu < 4; ++mu)
                        lub[((((size_t)zt * 4 + mu) * nb + b1) * nb + b2) * n_phib + kb] += T[mu];
                    lnb[(((size_t)zt * nb + b1) * nb + b2) * n_phib + kb] += www;
                    /* centroid projection from the q-vectors of this triplet */
                    const cplx v1 = dxj + I * dyj, v2 = dxk + I * dyk;
                    const cplx q1 = -(v1 + v2) / 3.0, q2 = (2.0 * v1 - v2) / 3.0, q3 = (2.0 * v2 - v1) / 3.0;
                    if (q1 == 0 || q2 == 0 || q3 == 0) continue;
                    cplx Tc[4];
                    Tc[0] = www * proj_cen(gi, q1, 0) * proj_cen(gj, q2, 0) * proj_cen(gk, q3, 0);
                    Tc[1] = www * proj_cen(gi, q1, 1) * proj_cen(gj, q2, 0) * proj_cen(gk, q3, 0);
                    Tc[2] = www * proj_cen(gi, q1, 0) * proj_cen(gj, q2, 1) * proj_cen(gk, q3, 0);
                    Tc[3] = www * proj_cen(gi, q1, 0) * proj_cen(gj, q2, 0) * proj_cen(gk, q3, 1);
                    const double t1 = cabs(v1), t2 = cabs(v2);
                    for (int mu = 0; mu < 4; ++mu) {
                        luc[((((size_t)zt * 4 + mu) * nb + b1) * nb + b2) * n_phib + kb] += Tc[mu];
                        const double d = cabs(Tc[mu] - T[mu] * cen_factor(mu, t1, t2, phi));
                        if (d > ldev) ldev = d;
                        if (cabs(T[mu]) > ltmax) ltmax = cabs(T[mu]);
                    }
                }
            }
        }
#pragma omp critical
        {
            for (size_t q = 0; q < s_un; ++q) ups_n[q] += lun[q];
            for (size_t q = 0; q < s_nn; ++q) norm_n[q] += lnn[q];
            for (size_t q = 0; q < s_ub; ++q) ups_b[q] += lub[q];
            for (size_t q = 0; q < s_nb; ++q) norm_b[q] += lnb[q];
            for (size_t q = 0; q < s_ub; ++q) upsc_b[q] += luc[q];
            if (ldev > dev) dev = ldev;
            if (ltmax > tmax) tmax = ltmax;
        }
        free(lun);
        free(lnn);
        free(lub);
        free(lnb);
        free(luc);
        free(nbr);
        free(nbb);
    }
    if (p5_dev) *p5_dev = tmax > 0 ? dev / tmax : 0;
    free(e2q);
    return ORC_OK;
}

/* ---- Direct estimator of the third-order aperture mass (Sec. 5.3, Eq. MapDirectEstimator) ----
 * At the aperture centre c (arcmin) and aperture radii (t1, t2, t3):
 *   num = sum over distinct i, j, k of w_i w_j w_k Q_t1(r_i) Q_t2(r_j) Q_t3(r_k) gt_i gt_j gt_k
 *   den = the same sum without the tangential shears,
 * with r_i = |x_i - c|, gt_i = Re(gamma(x_i; zeta_i)) the tangential shear about c (zeta_i the
 * polar angle of x_i - c, Eq. gammatx_def) and Q the filter of Eq. CrittendenQ,
 * Q_t(r) = r^2 / (4 pi t^4) exp(-r^2 / (2 t^2)); galaxies farther than rcut from c are left out.
 * The estimate at c is num / den; <M_ap^3> is its average over apertures. */

static double q_filter(double r, double t)
{
    return r * r / (4.0 * M_PI * t * t * t * t) * exp(-r * r / (2.0 * t * t));
}

/* the per-galaxy factors a_l = w Q_tl gt (with_gt) or w Q_tl, l = 0..2; 0 beyond rcut */
static int direct_factors(double x, double y, float g1, float g2, float w, double cx, double cy,
                          const double* th, double rcut, int with_gt, double a[3])
{
    const double dx = x - cx, dy = y - cy, r = sqrt(dx * dx + dy * dy);
    if (r > rcut || r == 0.0) {
        a[0] = a[1] = a[2] = 0.0;
        return 0;
    }
    double gt = 1.0;
    if (with_gt) gt = creal(proj((double)g1 + I * (double)g2, atan2(dy, dx), 0));
    for (int l = 0; l < 3; ++l) a[l] = (double)w * q_filter(r, th[l]) * gt;
    return 1;
}

/* Literal triple loop over distinct (i, j, k): the definition, for tiny catalogs. */
int orc_map3_direct_brute(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1,
                          const float* g2, const float* w, double quantum, double cx, double cy,
                          const double* th, double rcut, double* num, double* den)
{
    double sn = 0.0, sd = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ai[3], bi[3];
        direct_factors(xq[i] * quantum, yq[i] * quantum, g1[i], g2[i], w[i], cx, cy, th, rcut, 1, ai);
        direct_factors(xq[i] * quantum, yq[i] * quantum, g1[i], g2[i], w[i], cx, cy, th, rcut, 0, bi);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double aj[3], bj[3];
            direct_factors(xq[j] * quantum, yq[j] * quantum, g1[j], g2[j], w[j], cx, cy, th, rcut, 1, aj);
            direct_factors(xq[j] * quantum, yq[j] * quantum, g1[j], g2[j], w[j], cx, cy, th, rcut, 0, bj);
            for (int64_t k = 0; k < n; ++k) {
                if (k == i || k == j) continue;
                double ak[3], bk[3];
                direct_factors(xq[k] * quantum, yq[k] * quantum, g1[k], g2[k], w[k], cx, cy, th, rcut, 1, ak);
                direct_factors(xq[k] * quantum, yq[k] * quantum, g1[k], g2[k], w[k], cx, cy, th, rcut, 0, bk);
                sn += ai[0] * aj[1] * ak[2];
                sd += bi[0] * bj[1] * bk[2];
            }
        }
    }
    *num = sn;
    *den = sd;
    return ORC_OK;
}

/* The same sums for many apertures in O(n) each: for factors a, b, c of the three slots,
 *   sum_{i,j,k distinct} a_i b_j c_k = A B C - (AB) C - (AC) B - (BC) A + 2 (ABC)
 * (inclusion-exclusion over the coincidences i = j, i = k, j = k; A = sum a_i, AB = sum a_i b_i,
 * ...). out[t][0..1] = (num, den) of aperture t; centres [n_cen][2] arcmin. */
int orc_map3_direct(int64_t n, const int32_t* xq, const int32_t* yq, const float* g1, const float* g2,
                    const float* w, double quantum, int64_t n_cen, const double* centres,
                    const double* th, double rcut, double* out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_cen; ++t) {
        double s[2][7] = {{0}};
        for (int64_t i = 0; i < n; ++i) {
            for (int with_gt = 1; with_gt >= 0; --with_gt) {
                double a[3];
                if (!direct_factors(xq[i] * quantum, yq[i] * quantum, g1[i], g2[i], w[i], centres[2 * t],
                                    centres[2 * t + 1], th, rcut, with_gt, a))
                    break;
                double* q = s[1 - with_gt];
                q[0] += a[0];
                q[1] += a[1];
                q[2] += a[2];
                q[3] += a[0] * a[1];
                q[4] += a[0] * a[2];
                q[5] += a[1] * a[2];
                q[6] += a[0] * a[1] * a[2];
            }
        }
        for (int v = 0; v < 2; ++v) {
            const double* q = s[v];
            out[2 * t + v] = q[0] * q[1] * q[2] - q[3] * q[2] - q[4] * q[1] - q[5] * q[0] + 2.0 * q[6];
        }
    }
    return ORC_OK;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following parallel regions (timing on a given number of host cores) */
int orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
