/*
 * FP64 CPU oracle for the VSA-OGM hot path (arXiv 2408.09066).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * in __graft_entry__.py and the CPU-baseline leg of bench.py may load this
 * library.  It shares no code, header, table or constant generator with the
 * CUDA path; it is written from the paper's definitions, slowly and plainly,
 * in double precision, so that a reader can check each function against the
 * equation it cites.
 *
 * Conventions (readings of the paper where it is silent; each is listed in the
 * design notes):
 *   - FHRR form of the SSP encoding.  The Fourier coefficients of an axis
 *     vector are unit phasors e^{i theta_k}; raising them to the power x/l
 *     (Eq. fb-with-ls-1d, Eq. fb-with-ls-2d) gives phi_k(x, y) =
 *     exp(i 2 pi (nu_x[k] x + nu_y[k] y)), where nu = theta / (2 pi l) is a
 *     frequency in cycles per metre.  The length scale l is folded into nu.
 *   - nu is drawn uniformly from (-1/(2l), 1/(2l)) (theta uniform on
 *     (-pi, pi)) with SplitMix64 and stored as float32 by definition.
 *   - Similarity (Eq. loc-query) is Re <omega, phi> = Re sum_k conj(omega_k) phi_k.
 *   - Tiles are numbered beta = by * tiles_x + bx; memory index is 2 beta + psi
 *     (Algorithm 1).
 *   - Cell (i, j) has centre (x_min + (i + 1/2) res, y_min + (j + 1/2) res).
 *   - 0 ln 0 := 0; natural logarithm.
 *   - A class whose map maximum is <= 0 decodes to all zeros.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586476925286766559

/* Grid description, owned by this file (the CUDA library has its own). */
typedef struct {
    int32_t W, H;        /* cells along x and y */
    double res;          /* cell edge length in metres */
    double x_min, y_min; /* lower-left corner of the map */
    int32_t tiles_x;     /* delta along x */
    int32_t tiles_y;     /* delta along y */
} orc_grid;

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the parallel loops below use (1 without OpenMP). */
int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio gamma
 * 0x9E3779B97F4A7C15 and each state is passed through the variant-13 mixer.
 * Written as a counter-based generator: output number i (0-based) of the
 * stream seeded with `seed` is mix(seed + (i + 1) * gamma).                  */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Axis vectors (Initialization, Sec. III-B2): D frequencies per axis.
 * u = top 53 bits of the output / 2^53 in [0, 1); nu = f32((2u - 1) * 0.5 / l).
 * nu_x[k] uses output 2k and nu_y[k] output 2k + 1, so a longer vector
 * extends a shorter one with the same seed.                                  */
void orc_draw_nu(uint64_t seed, int32_t D, double length_scale, float *nu_x, float *nu_y)
{
    for (int32_t k = 0; k < D; ++k) {
        double ux = (double)(orc_splitmix64_at(seed, 2u * (uint64_t)k) >> 11) * 0x1.0p-53;
        double uy = (double)(orc_splitmix64_at(seed, 2u * (uint64_t)k + 1u) >> 11) * 0x1.0p-53;
        nu_x[k] = (float)((2.0 * ux - 1.0) * (0.5 / length_scale));
        nu_y[k] = (float)((2.0 * uy - 1.0) * (0.5 / length_scale));
    }
}

/* ------------------------------------------------------------------------ */
/* Tiling (Sec. III-B3): delta evenly sized tiles per axis. */
static double tile_w(const orc_grid *g) { return (double)g->W * g->res / (double)g->tiles_x; }
static double tile_h(const orc_grid *g) { return (double)g->H * g->res / (double)g->tiles_y; }

void orc_tile_centre(const orc_grid *g, int32_t beta, double *cx, double *cy)
{
    int32_t bx = beta % g->tiles_x, by = beta / g->tiles_x;
    *cx = g->x_min + ((double)bx + 0.5) * tile_w(g);
    *cy = g->y_min + ((double)by + 0.5) * tile_h(g);
}

/* Algorithm 1: beta = argmin_k d_L2(gamma, mu_k); the first minimum wins. */
int32_t orc_tile_of(const orc_grid *g, double x, double y)
{
    int32_t T = g->tiles_x * g->tiles_y, best = 0;
    double best_d2 = INFINITY;
    for (int32_t k = 0; k < T; ++k) {
        double cx, cy;
        orc_tile_centre(g, k, &cx, &cy);
        double d2 = (x - cx) * (x - cx) + (y - cy) * (y - cy);
        if (d2 < best_d2) { best_d2 = d2; best = k; }
    }
    return best;
}

void orc_assign(const orc_grid *g, const float *xy, int64_t n, int32_t *beta)
{
    for (int64_t p = 0; p < n; ++p) beta[p] = orc_tile_of(g, xy[2 * p], xy[2 * p + 1]);
}

/* ------------------------------------------------------------------------ */
/* Encoding and bundling (Eq. fb-with-ls-2d, Eq. bundling, Algorithm 1).
 * omega has layout [2T][D][2] (re, im) with memory index 2 beta + psi.
 * frame = 0: global coordinates, phi_k(p) = exp(i 2 pi (nu_x p_x + nu_y p_y)).
 * frame = 1: tile-centred coordinates p - mu_beta, which multiplies memory
 *            2 beta + psi by the unit phasor exp(-i 2 pi nu . mu_beta).
 * Only the k listed in ks[0..nk) are computed (ks == NULL: all k < D); the
 * output then has layout [2T][nk][2].  Returns -1 on a label outside {0,1}. */
int32_t orc_memories(const orc_grid *g, int32_t D, const float *nu_x, const float *nu_y,
                     const float *xy, const uint8_t *labels, int64_t n, int32_t frame,
                     const int32_t *ks, int32_t nk, const int32_t *beta_in, double *omega)
{
    int32_t T = g->tiles_x * g->tiles_y;
    if (ks == NULL) nk = D;
    for (int64_t p = 0; p < n; ++p)
        if (labels[p] > 1) return -1;
    int32_t *beta = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    /* beta_in: the caller's exact tile assignment (see oracle.assign); else FP64 argmin */
    if (beta_in)
        memcpy(beta, beta_in, sizeof(int32_t) * (size_t)n);
    else
        orc_assign(g, xy, n, beta);
    memset(omega, 0, sizeof(double) * (size_t)2 * T * nk * 2);
#pragma omp parallel for schedule(static)
    for (int32_t q = 0; q < nk; ++q) {
        int32_t k = ks ? ks[q] : q;
        for (int64_t p = 0; p < n; ++p) {
            double x = (double)xy[2 * p], y = (double)xy[2 * p + 1];
            if (frame == 1) {
                double cx, cy;
                orc_tile_centre(g, beta[p], &cx, &cy);
                x -= cx;
                y -= cy;
            }
            double turns = (double)nu_x[k] * x + (double)nu_y[k] * y;
            double ph = ORC_TWO_PI * turns;
            size_t m = (size_t)(2 * beta[p] + labels[p]);
            omega[(m * nk + q) * 2 + 0] += cos(ph);
            omega[(m * nk + q) * 2 + 1] += sin(ph);
        }
    }
    free(beta);
    return 0;
}

/* Eq. vector-normalization: ||omega_m|| for each of the nmem memories. */
void orc_norms(const double *omega, int32_t nmem, int32_t D, double *norms)
{
    for (int32_t m = 0; m < nmem; ++m) {
        double s = 0.0;
        for (int32_t k = 0; k < D; ++k) {
            double re = omega[((size_t)m * D + k) * 2], im = omega[((size_t)m * D + k) * 2 + 1];
            s += re * re + im * im;
        }
        norms[m] = sqrt(s);
    }
}

/* Eq. loc-query after Eq. vector-normalization, memory-vector form, for the
 * cells listed as (i, j) pairs: P[c][psi] = Re sum_k conj(w_k) phi_k(cell) / ||w||
 * with w the memory of the cell's tile and class psi.  The cell's tile is
 * chosen by Algorithm 1's rule applied to the cell centre; `frame` must match
 * the frame the memories were built in.                                      */
void orc_decode_cells(const orc_grid *g, int32_t D, const float *nu_x, const float *nu_y,
                      const double *omega, int32_t frame, const int32_t *cells, int64_t ncells,
                      const int32_t *beta_cells, double *P)
{
    int32_t T = g->tiles_x * g->tiles_y;
    double *norms = (double *)malloc(sizeof(double) * 2 * T);
    orc_norms(omega, 2 * T, D, norms);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < ncells; ++c) {
        double x = g->x_min + ((double)cells[2 * c] + 0.5) * g->res;
        double y = g->y_min + ((double)cells[2 * c + 1] + 0.5) * g->res;
        int32_t beta = beta_cells ? beta_cells[c] : orc_tile_of(g, x, y);
        if (frame == 1) {
            double cx, cy;
            orc_tile_centre(g, beta, &cx, &cy);
            x -= cx;
            y -= cy;
        }
        for (int32_t psi = 0; psi < 2; ++psi) {
            size_t m = (size_t)(2 * beta + psi);
            double acc = 0.0;
            for (int32_t k = 0; k < D; ++k) {
                double ph = ORC_TWO_PI * ((double)nu_x[k] * x + (double)nu_y[k] * y);
                double wr = omega[(m * D + k) * 2], wi = omega[(m * D + k) * 2 + 1];
                /* Re(conj(w) * e^{i ph}) = wr cos(ph) + wi sin(ph) */
                acc += wr * cos(ph) + wi * sin(ph);
            }
            P[2 * c + psi] = norms[m] > 0.0 ? acc / norms[m] : 0.0;
        }
    }
    free(norms);
}

/* The whole map: P has layout [2][H][W] (class, row j, column i).  beta_cells
 * (nullable) gives the tile of each cell in the same row-major order.      */
void orc_decode_map(const orc_grid *g, int32_t D, const float *nu_x, const float *nu_y,
                    const double *omega, int32_t frame, const int32_t *beta_cells, double *P)
{
    int64_t nc = (int64_t)g->W * g->H;
    int32_t *cells = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)nc);
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)nc);
    for (int64_t c = 0; c < nc; ++c) {
        cells[2 * c] = (int32_t)(c % g->W);
        cells[2 * c + 1] = (int32_t)(c / g->W);
    }
    orc_decode_cells(g, D, nu_x, nu_y, omega, frame, cells, nc, beta_cells, tmp);
    for (int64_t c = 0; c < nc; ++c) {
        P[c] = tmp[2 * c];
        P[nc + c] = tmp[2 * c + 1];
    }
    free(cells);
    free(tmp);
}

/* The direct per-cell sum over points, with no memory vector at all:
 *   numerator   = sum_{p in (beta, psi)} sum_k cos(2 pi nu_k . (cell - p))
 *   ||omega||^2 = sum_{p, q in (beta, psi)} sum_k cos(2 pi nu_k . (p - q))
 * This is Eq. loc-query expanded through Eq. bundling; it is independent of
 * the frame.  Cost is O(n^2 D): tiny inputs only.                          */
void orc_direct_cells(const orc_grid *g, int32_t D, const float *nu_x, const float *nu_y,
                      const float *xy, const uint8_t *labels, int64_t n,
                      const int32_t *cells, int64_t ncells, const int32_t *beta_in,
                      const int32_t *beta_cells, double *P)
{
    int32_t T = g->tiles_x * g->tiles_y;
    int32_t *beta = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *norm2 = (double *)calloc((size_t)2 * T, sizeof(double));
    if (beta_in)
        memcpy(beta, beta_in, sizeof(int32_t) * (size_t)n);
    else
        orc_assign(g, xy, n, beta);
    for (int64_t p = 0; p < n; ++p)
        for (int64_t q = 0; q < n; ++q) {
            if (beta[p] != beta[q] || labels[p] != labels[q]) continue;
            double dx = (double)xy[2 * p] - (double)xy[2 * q];
            double dy = (double)xy[2 * p + 1] - (double)xy[2 * q + 1];
            double s = 0.0;
            for (int32_t k = 0; k < D; ++k)
                s += cos(ORC_TWO_PI * ((double)nu_x[k] * dx + (double)nu_y[k] * dy));
            norm2[2 * beta[p] + labels[p]] += s;
        }
    for (int64_t c = 0; c < ncells; ++c) {
        double x = g->x_min + ((double)cells[2 * c] + 0.5) * g->res;
        double y = g->y_min + ((double)cells[2 * c + 1] + 0.5) * g->res;
        int32_t b = beta_cells ? beta_cells[c] : orc_tile_of(g, x, y);
        for (int32_t psi = 0; psi < 2; ++psi) {
            double num = 0.0;
            for (int64_t p = 0; p < n; ++p) {
                if (beta[p] != b || labels[p] != psi) continue;
                double dx = x - (double)xy[2 * p], dy = y - (double)xy[2 * p + 1];
                for (int32_t k = 0; k < D; ++k)
                    num += cos(ORC_TWO_PI * ((double)nu_x[k] * dx + (double)nu_y[k] * dy));
            }
            double nm = norm2[2 * b + psi];
            P[2 * c + psi] = nm > 0.0 ? num / sqrt(nm) : 0.0;
        }
    }
    free(beta);
    free(norm2);
}

/* ------------------------------------------------------------------------ */
/* Eq. non-linearities: P_hat = (P / max(P))^2 per class over the whole map.
 * P and Phat have layout [2][ncell]; maxima receives max(P) per class.       */
void orc_nonlinear(const double *P, int64_t ncell, double *Phat, double *maxima)
{
    for (int32_t c = 0; c < 2; ++c) {
        double m = -INFINITY;
        for (int64_t q = 0; q < ncell; ++q) m = P[c * ncell + q] > m ? P[c * ncell + q] : m;
        maxima[c] = m;
        for (int64_t q = 0; q < ncell; ++q) {
            double v = m > 0.0 ? P[c * ncell + q] / m : 0.0;
            Phat[c * ncell + q] = v * v;
        }
    }
}

/* Algorithm 2 with the localized Shannon entropy and the disk mask
 * (Eq. entropy-mask): H(x, y) = - sum over in-grid (x', y') with
 * (x'-x)^2 + (y'-y)^2 <= r^2 of P log P, natural log, 0 log 0 = 0.  The
 * summand is taken as 0 for P < 0, which only the decoding ablation without
 * the squaring step can produce (P_hat is a square otherwise).
 * Distances are in cell units.  Phat and Hout are one class map each, layout
 * [H][W].                                                                    */
void orc_entropy(const double *Phat, int32_t W, int32_t H, int32_t r, double *Hout)
{
#pragma omp parallel for schedule(static)
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            double s = 0.0;
            /* cells outside the (2r+1)^2 box around (x, y) are farther than r */
            int32_t y0 = y - r < 0 ? 0 : y - r, y1 = y + r > H - 1 ? H - 1 : y + r;
            int32_t x0 = x - r < 0 ? 0 : x - r, x1 = x + r > W - 1 ? W - 1 : x + r;
            for (int32_t yy = y0; yy <= y1; ++yy)
                for (int32_t xx = x0; xx <= x1; ++xx) {
                    int64_t d2 = (int64_t)(xx - x) * (xx - x) + (int64_t)(yy - y) * (yy - y);
                    if (d2 > (int64_t)r * r) continue;
                    double v = Phat[(size_t)yy * W + xx];
                    if (v > 0.0) s -= v * log(v); /* 0 ln 0 = 0; v < 0 carries no mass */
                }
            Hout[(size_t)y * W + x] = s;
        }
}

/* Eq. softmax over the two classes and Eq. psd:
 * Pr(psi) = e^{H_psi} / (e^{H_0} + e^{H_1}); OGM = Pr(1) - Pr(0).
 * The common factor e^{-max(H_0, H_1)} is taken out of numerator and
 * denominator, which leaves the value unchanged and avoids overflow.         */
void orc_softmax_psd(const double *H0, const double *H1, int64_t n, double *pr1, double *pr0,
                     double *ogm)
{
    for (int64_t q = 0; q < n; ++q) {
        double m = H0[q] > H1[q] ? H0[q] : H1[q];
        double e0 = exp(H0[q] - m), e1 = exp(H1[q] - m);
        pr1[q] = e1 / (e0 + e1);
        pr0[q] = e0 / (e0 + e1);
        ogm[q] = pr1[q] - pr0[q];
    }
}

/* Eq. classification, decided in float32 on float32 inputs:
 * occupied (1) iff OGM >= rho.                                              */
void orc_classify_f32(const float *ogm, int64_t n, float rho, uint8_t *cls)
{
    for (int64_t q = 0; q < n; ++q) cls[q] = (uint8_t)(ogm[q] >= rho ? 1 : 0);
}
