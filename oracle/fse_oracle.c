/*
 * fse_oracle.c -- plain, slow FP64 CPU oracle for Frequency Selective
 * Extrapolation (FSE) on the overlapping tiles of the paper's tiling algorithm.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product library never
 * links, includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   1. Tiling, Algorithm 1 with Eqs. (1)-(4) (Sec. III): aspect ratio r = W/H,
 *      rows n_R = max(1, round(sqrt(N/r))), tiles per row n_C, row height h_T,
 *      tile width w_T; the last row takes the remaining height.  Landscape is
 *      assumed; a portrait image is tiled with its axes swapped (Sec. III).
 *   2. Each tile is extended by a stripe of d pixels on every side (Sec. III,
 *      "a stripe of d samples width"), clipped to the image.  Every extended
 *      tile is extrapolated as a standalone image by the unchanged algorithm.
 *   3. FSE per extended tile (Sec. II): the tile is cut into b x b blocks; each
 *      block containing a lost pixel is modelled from its (b+2B)^2 support as a
 *      sparse weighted sum of F x F Fourier basis functions, chosen greedily:
 *        w   = rho^dist on known pixels, delta*rho^dist on pixels reconstructed
 *              by earlier blocks, 0 on pending (lost, not yet reconstructed)
 *              pixels and outside the extended tile;
 *        per iteration: p_k = sum w r exp(-2 pi i k.x/F) for every bin k
 *              (explicit spatial-domain projections, no FFT, no spectral
 *              update), u = argmax |p_k|^2, Delta = gamma p_u / sum(w),
 *              c_u += Delta, r -= Delta phi_u with phi_u = exp(+2 pi i u.x/F);
 *        the model Re sum_u c_u phi_u fills the block's pending pixels.
 *   4. Crop and merge (Sec. III): each output pixel comes from the tile whose
 *      core contains it; known pixels are copied.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - n_R uses round-half-up evaluated in exact integers.
 *   - Degenerate tiles (w_T <= 0 or h_T <= 0) are an error, not "fixed".
 *   - Block grid origin = the extended tile's top-left; a block is lost if it
 *     holds at least one lost pixel; its known pixels stay known.
 *   - Processing order: PHASED (P = ceil(B/b)+1, key ((I mod P)P + J mod P, I, J)),
 *     RASTER (I, J) or INDEPENDENT (earlier reconstructions are never used).
 *   - Weight centre m_c = n_c = B + (b-1)/2; delta multiplies rho^dist.
 *   - Argmax tie rule: the lowest flat index k1*F+k2 among
 *     |p_k|^2 >= (1-tau) max |p|^2.
 *   - Output u8 = round-half-even(clip(g, 0, 255)); g is stored unrounded.
 *   - sum(w) == 0: no iteration, the block's pixels stay pending, output 0.
 */
#include <complex.h>
#undef I /* block-grid indices are called I, J below */
#define IU _Complex_I
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EDEGENERATE (-2)
#define OR_ENOMEM (-3)

#define ORDER_PHASED 0
#define ORDER_RASTER 1
#define ORDER_INDEPENDENT 2

#define ST_KNOWN 0
#define ST_PENDING 1
#define ST_DONE 2

/* ------------------------------------------------------------------------ */
/* 1. Tiling: Algorithm 1, Eqs. (1)-(4).                                    */
/* ------------------------------------------------------------------------ */

/* Eq. (2): n_R = max(1, round(sqrt(N / r))) with r = W/H (Eq. 1).
 * sqrt(N H / W) rounded half up equals the largest n >= 1 with
 * (n - 1/2)^2 <= N H / W, i.e. (2n-1)^2 W <= 4 N H; none means round() gave 0. */
static int64_t rows_eq2(int64_t W, int64_t H, int64_t N) {
    int64_t n = 0;
    while ((2 * (n + 1) - 1) * (2 * (n + 1) - 1) * W <= 4 * N * H) n++;
    return n < 1 ? 1 : n;
}

/* Writes N tiles as 8 int32 each: x, y, w, h (core) and ex, ey, ew, eh
 * (core grown by d on every side, clipped to the image). */
int oracle_plan_tiles(int32_t W32, int32_t H32, int32_t N32, int32_t d32,
                      int32_t *out, int32_t cap, int32_t *n_out) {
    if (n_out) *n_out = 0;
    if (W32 <= 0 || H32 <= 0 || N32 <= 0 || d32 < 0) return OR_EINVAL;
    if (cap < N32) return OR_EINVAL;
    int swap = W32 < H32; /* landscape assumed; otherwise swap the axes */
    int64_t W = swap ? H32 : W32, H = swap ? W32 : H32, N = N32, d = d32;
    int64_t nR = rows_eq2(W, H, N);
    int64_t yT = 0;
    int32_t t = 0;
    for (int64_t i = 1; i <= nR; i++) {
        /* Eq. (3): tiles in row i */
        int64_t nC = (i <= N % nR) ? (N + nR - 1) / nR : N / nR;
        /* Eq. (4): row height; the last row covers the rest of the image */
        int64_t hT = (H * nC) / N + ((H * nC) % N) / nR;
        if (i == nR) hT = H - yT;
        int64_t xT = 0;
        for (int64_t j = 1; j <= nC; j++) {
            /* Eq. (5): tile width */
            int64_t wT = (j <= W % nC) ? (W + nC - 1) / nC : W / nC;
            if (wT <= 0 || hT <= 0) return OR_EDEGENERATE;
            int64_t ex0 = xT - d < 0 ? 0 : xT - d;
            int64_t ey0 = yT - d < 0 ? 0 : yT - d;
            int64_t ex1 = xT + wT + d > W ? W : xT + wT + d;
            int64_t ey1 = yT + hT + d > H ? H : yT + hT + d;
            int32_t *o = out + 8 * t;
            if (!swap) {
                o[0] = (int32_t)xT; o[1] = (int32_t)yT; o[2] = (int32_t)wT; o[3] = (int32_t)hT;
                o[4] = (int32_t)ex0; o[5] = (int32_t)ey0;
                o[6] = (int32_t)(ex1 - ex0); o[7] = (int32_t)(ey1 - ey0);
            } else {
                o[0] = (int32_t)yT; o[1] = (int32_t)xT; o[2] = (int32_t)hT; o[3] = (int32_t)wT;
                o[4] = (int32_t)ey0; o[5] = (int32_t)ex0;
                o[6] = (int32_t)(ey1 - ey0); o[7] = (int32_t)(ex1 - ex0);
            }
            t++;
            xT += wT;
        }
        yT += hT;
    }
    if (t != N) return OR_EDEGENERATE; /* cannot happen: sum of n_C is N */
    if (n_out) *n_out = t;
    return OR_OK;
}

/* The comparison tiling of Sec. III: N vertical stripes of full height,
 * widths floor(W/N) with the first W mod N one wider (the Eq. 5 rule). */
int oracle_plan_vertical(int32_t W, int32_t H, int32_t N, int32_t d, int32_t *out, int32_t cap,
                         int32_t *n_out) {
    if (n_out) *n_out = 0;
    if (W <= 0 || H <= 0 || N <= 0 || d < 0 || cap < N) return OR_EINVAL;
    int64_t x = 0;
    for (int j = 1; j <= N; j++) {
        int64_t w = W / N + (j <= W % N ? 1 : 0);
        if (w <= 0) return OR_EDEGENERATE;
        int64_t x0 = x - d < 0 ? 0 : x - d, x1 = x + w + d > W ? W : x + w + d;
        int32_t *o = out + 8 * (j - 1);
        o[0] = (int32_t)x; o[1] = 0; o[2] = (int32_t)w; o[3] = H;
        o[4] = (int32_t)x0; o[5] = 0; o[6] = (int32_t)(x1 - x0); o[7] = H;
        x += w;
    }
    if (n_out) *n_out = N;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 2. FSE on one block's support (Sec. II): greedy weighted model fit.      */
/* ------------------------------------------------------------------------ */

/* p[k1*F+k2] = sum_{m,n<S} v[m*S+n] exp(-2 pi i (k1 m + k2 n)/F), evaluated as
 * two explicit direct sums (first over n, then over m). tw[q] = exp(-2 pi i q/F). */
static void project(const double complex *v, int S, int F, const double complex *tw,
                    double complex *A /* S*F */, double complex *p /* F*F */) {
    for (int m = 0; m < S; m++)
        for (int k2 = 0; k2 < F; k2++) {
            double complex s = 0;
            for (int n = 0; n < S; n++) s += v[m * S + n] * tw[(k2 * n) % F];
            A[m * F + k2] = s;
        }
    for (int k1 = 0; k1 < F; k1++)
        for (int k2 = 0; k2 < F; k2++) {
            double complex s = 0;
            for (int m = 0; m < S; m++) s += A[m * F + k2] * tw[(k1 * m) % F];
            p[k1 * F + k2] = s;
        }
}

static void twiddles(int F, double complex *tw) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int q = 0; q < F; q++) tw[q] = cos(two_pi * q / F) - IU * sin(two_pi * q / F);
}

/*
 * Greedy fit of one support (S x S, row-major, m = row, n = column).
 *   w      : weights (>= 0)
 *   r_re/im: initial residual r^0 (the signal; zero where w == 0 is fine)
 * Outputs (any may be NULL except c_re/c_im):
 *   useq[K]          selected bin u (flat k1*F+k2) per iteration
 *   c_re/c_im[F*F]   accumulated coefficients c_u
 *   energy[K+1]      weighted residual energy sum w |r|^2 before each
 *                    iteration and after the last one
 *   r_out_re/im[S*S] final residual
 * Returns W0 = sum w; when W0 == 0 nothing is iterated (c stays 0).
 */
double oracle_fse_fit(const double *w, const double *r_re, const double *r_im, int S, int F,
                      int K, double gamma, double tau, int32_t *useq, double *c_re, double *c_im,
                      double *energy, double *r_out_re, double *r_out_im) {
    double W0 = 0;
    for (int i = 0; i < S * S; i++) W0 += w[i];
    for (int i = 0; i < F * F; i++) { c_re[i] = 0; c_im[i] = 0; }
    double complex *tw = malloc(sizeof(double complex) * F);
    double complex *r = malloc(sizeof(double complex) * S * S);
    double complex *v = malloc(sizeof(double complex) * S * S);
    double complex *A = malloc(sizeof(double complex) * S * F);
    double complex *p = malloc(sizeof(double complex) * F * F);
    twiddles(F, tw);
    for (int i = 0; i < S * S; i++) r[i] = r_re[i] + IU * (r_im ? r_im[i] : 0.0);
    if (W0 > 0) {
        for (int it = 0; it < K; it++) {
            if (energy) {
                double e = 0;
                for (int i = 0; i < S * S; i++) e += w[i] * (creal(r[i]) * creal(r[i]) + cimag(r[i]) * cimag(r[i]));
                energy[it] = e;
            }
            /* weighted residual spectrum, explicit projections */
            for (int i = 0; i < S * S; i++) v[i] = w[i] * r[i];
            project(v, S, F, tw, A, p);
            /* selection: largest |p_k|^2, lowest flat index among near-ties */
            double emax = -1;
            for (int k = 0; k < F * F; k++) {
                double e = creal(p[k]) * creal(p[k]) + cimag(p[k]) * cimag(p[k]);
                if (e > emax) emax = e;
            }
            int u = 0;
            for (int k = 0; k < F * F; k++) {
                double e = creal(p[k]) * creal(p[k]) + cimag(p[k]) * cimag(p[k]);
                if (e >= (1.0 - tau) * emax) { u = k; break; }
            }
            if (useq) useq[it] = u;
            /* coefficient update and residual update with the same Delta */
            double complex delta = gamma * p[u] / W0;
            c_re[u] += creal(delta);
            c_im[u] += cimag(delta);
            int u1 = u / F, u2 = u % F;
            for (int m = 0; m < S; m++)
                for (int n = 0; n < S; n++) {
                    /* phi_u(m,n) = exp(+2 pi i (u1 m + u2 n)/F) = conj(tw[...]) */
                    double complex phi = conj(tw[(u1 * m + u2 * n) % F]);
                    r[m * S + n] -= delta * phi;
                }
        }
        if (energy) {
            double e = 0;
            for (int i = 0; i < S * S; i++) e += w[i] * (creal(r[i]) * creal(r[i]) + cimag(r[i]) * cimag(r[i]));
            energy[K] = e;
        }
    }
    if (r_out_re)
        for (int i = 0; i < S * S; i++) { r_out_re[i] = creal(r[i]); if (r_out_im) r_out_im[i] = cimag(r[i]); }
    free(tw); free(r); free(v); free(A); free(p);
    return W0;
}

/* Model value g(m,n) = Re sum_u c_u exp(+2 pi i (u1 m + u2 n)/F). */
double oracle_fse_model(const double *c_re, const double *c_im, int F, int m, int n) {
    const double two_pi = 6.283185307179586476925286766559;
    double g = 0;
    for (int u1 = 0; u1 < F; u1++)
        for (int u2 = 0; u2 < F; u2++) {
            int k = u1 * F + u2;
            if (c_re[k] == 0 && c_im[k] == 0) continue;
            int q = (u1 * m + u2 * n) % F;
            g += c_re[k] * cos(two_pi * q / F) - c_im[k] * sin(two_pi * q / F);
        }
    return g;
}

/* ------------------------------------------------------------------------ */
/* 3. Whole image: tiles, block order, staging, write-back, crop and merge. */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t I, J;      /* block row / column in the tile-local grid */
    int64_t key0;      /* first component of the order key */
} blk_t;

static int blk_cmp(const void *a, const void *b) {
    const blk_t *x = a, *y = b;
    if (x->key0 != y->key0) return x->key0 < y->key0 ? -1 : 1;
    if (x->I != y->I) return x->I < y->I ? -1 : 1;
    if (x->J != y->J) return x->J < y->J ? -1 : 1;
    return 0;
}

/* One processed block as reported to the caller (for selection-sequence checks). */
typedef struct {
    int32_t tile, I, J, status; /* status 1 = modelled, 2 = empty support */
    double W0;
} blk_report_t;

static double rint_half_even(double x) { return nearbyint(x); }

/*
 * Extrapolates one 8-bit image.  mask != 0 marks a lost pixel.
 *   params: b (block), B (border), F (DFT size), K, rho, delta, gamma,
 *           order, N (tiles), d (overlap), tau (tie tolerance)
 *   out[W*H]      : output image (u8)
 *   out_g[W*H]    : unrounded model value at lost pixels, NaN elsewhere (may be NULL)
 *   rep/useq      : optional per-block report (cap blocks; useq holds K ints each)
 *   nthreads      : OpenMP threads for blocks of one phase (<= 0: default)
 *   literal_seq   : 1 = strictly one block after another, each committed at once;
 *                   0 = blocks of one phase run concurrently and commit together
 *   max_blocks    : stop after this many blocks (<= 0: no limit); timing samples only
 *   stats[4]      : processed blocks, empty-support blocks, tiles, core lost blocks
 */
int oracle_fse_image(const uint8_t *img, const uint8_t *mask, int32_t W, int32_t H,
                     int32_t b, int32_t B, int32_t F, int32_t K, double rho, double delta,
                     double gamma, int32_t order, int32_t N, int32_t d, double tau,
                     uint8_t *out, double *out_g, blk_report_t *rep, int32_t *useq,
                     int32_t rep_cap, int32_t *n_rep, int32_t nthreads, int32_t literal_seq,
                     int64_t max_blocks, int64_t *stats, int32_t tiling) {
    if (n_rep) *n_rep = 0;
    if (b <= 0 || B < 0 || K < 0 || F <= 0) return OR_EINVAL;
    const int S = b + 2 * B;
    if (F < S) return OR_EINVAL;
    if (!(rho > 0 && rho <= 1) || !(gamma > 0 && gamma < 2) || delta < 0) return OR_EINVAL;
    if (order < 0 || order > 2) return OR_EINVAL;
    int32_t *tiles = malloc(sizeof(int32_t) * 8 * (size_t)(N > 0 ? N : 1));
    int32_t nt = 0;
    int rc = tiling == 1 ? oracle_plan_vertical(W, H, N, d, tiles, N, &nt)
                         : oracle_plan_tiles(W, H, N, d, tiles, N, &nt);
    if (rc != OR_OK) { free(tiles); return rc; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int64_t i = 0; i < (int64_t)W * H; i++) {
        out[i] = mask[i] ? 0 : img[i];
        if (out_g) out_g[i] = NAN;
    }
    /* isotropic weight: rho^dist about the block centre (B + (b-1)/2, same both axes) */
    double *wiso = malloc(sizeof(double) * S * S);
    const double mc = B + (b - 1) / 2.0;
    for (int m = 0; m < S; m++)
        for (int n = 0; n < S; n++)
            wiso[m * S + n] = pow(rho, sqrt((m - mc) * (m - mc) + (n - mc) * (n - mc)));
    const int P = (B + b - 1) / b + 1;
    int64_t n_proc = 0, n_empty = 0, n_core_lost = 0;
    int32_t nrep = 0;
    int stop = 0;

    for (int t = 0; t < nt && !stop; t++) {
        const int32_t cx = tiles[8 * t], cy = tiles[8 * t + 1], cw = tiles[8 * t + 2], ch = tiles[8 * t + 3];
        const int32_t ex = tiles[8 * t + 4], ey = tiles[8 * t + 5], ew = tiles[8 * t + 6], eh = tiles[8 * t + 7];
        /* the extended tile as a standalone image: value and state planes */
        double *val = malloc(sizeof(double) * (size_t)ew * eh);
        uint8_t *st = malloc((size_t)ew * eh);
        for (int y = 0; y < eh; y++)
            for (int x = 0; x < ew; x++) {
                int64_t gi = (int64_t)(ey + y) * W + (ex + x);
                st[y * ew + x] = mask[gi] ? ST_PENDING : ST_KNOWN;
                val[y * ew + x] = mask[gi] ? 0.0 : (double)img[gi];
            }
        const int nby = (eh + b - 1) / b, nbx = (ew + b - 1) / b;
        blk_t *bl = malloc(sizeof(blk_t) * (size_t)nby * nbx);
        int nb = 0;
        for (int I = 0; I < nby; I++)
            for (int J = 0; J < nbx; J++) {
                int lost = 0, core = 0;
                for (int y = I * b; y < (I + 1) * b && y < eh; y++)
                    for (int x = J * b; x < (J + 1) * b && x < ew; x++)
                        if (st[y * ew + x] == ST_PENDING) {
                            lost = 1;
                            int gx = ex + x, gy = ey + y;
                            if (gx >= cx && gx < cx + cw && gy >= cy && gy < cy + ch) core = 1;
                        }
                if (!lost) continue;
                n_core_lost += core;
                bl[nb].I = I;
                bl[nb].J = J;
                bl[nb].key0 = order == ORDER_PHASED ? (int64_t)(I % P) * P + (J % P) : 0;
                nb++;
            }
        qsort(bl, nb, sizeof(blk_t), blk_cmp);

        /* groups of blocks that may run together: one phase (PHASED), one block
         * (RASTER), everything (INDEPENDENT); literal_seq forces single blocks */
        int g0 = 0;
        while (g0 < nb && !stop) {
            int g1 = g0 + 1;
            if (!literal_seq) {
                if (order == ORDER_PHASED)
                    while (g1 < nb && bl[g1].key0 == bl[g0].key0) g1++;
                else if (order == ORDER_INDEPENDENT)
                    g1 = nb;
            }
            if (max_blocks > 0 && n_proc + (g1 - g0) > max_blocks) {
                g1 = g0 + (int)(max_blocks - n_proc);
                stop = 1;
            }
            const int ng = g1 - g0;
            double *gbuf = malloc(sizeof(double) * (size_t)ng * b * b);
            int32_t *gstat = malloc(sizeof(int32_t) * ng);
            double *gw0 = malloc(sizeof(double) * ng);
            int32_t *gseq = malloc(sizeof(int32_t) * (size_t)ng * (K > 0 ? K : 1));
            memset(gseq, 0xFF, sizeof(int32_t) * (size_t)ng * (K > 0 ? K : 1)); /* -1: not iterated */

#pragma omp parallel for schedule(dynamic)
            for (int q = 0; q < ng; q++) {
                const int I = bl[g0 + q].I, J = bl[g0 + q].J;
                double *w = malloc(sizeof(double) * S * S);
                double *r = malloc(sizeof(double) * S * S);
                double *cre = malloc(sizeof(double) * F * F);
                double *cim = malloc(sizeof(double) * F * F);
                /* support frame: tile-local rows I*b-B .., columns J*b-B .. */
                for (int m = 0; m < S; m++)
                    for (int n = 0; n < S; n++) {
                        int y = I * b - B + m, x = J * b - B + n;
                        double wv = 0, rv = 0;
                        if (y >= 0 && y < eh && x >= 0 && x < ew) {
                            int s = st[y * ew + x];
                            if (s == ST_KNOWN) { wv = wiso[m * S + n]; rv = val[y * ew + x]; }
                            else if (s == ST_DONE && order != ORDER_INDEPENDENT) {
                                wv = delta * wiso[m * S + n]; rv = val[y * ew + x];
                            }
                        }
                        w[m * S + n] = wv;
                        r[m * S + n] = rv;
                    }
                double W0 = oracle_fse_fit(w, r, NULL, S, F, K, gamma, tau, gseq + (size_t)q * K,
                                           cre, cim, NULL, NULL, NULL);
                gw0[q] = W0;
                gstat[q] = W0 > 0 ? 1 : 2;
                for (int yy = 0; yy < b; yy++)
                    for (int xx = 0; xx < b; xx++)
                        gbuf[(size_t)q * b * b + yy * b + xx] =
                            W0 > 0 ? oracle_fse_model(cre, cim, F, B + yy, B + xx) : 0.0;
                free(w); free(r); free(cre); free(cim);
            }

            /* commit: mark pending pixels done, write core pixels of the output */
            for (int q = 0; q < ng; q++) {
                const int I = bl[g0 + q].I, J = bl[g0 + q].J;
                for (int yy = 0; yy < b; yy++)
                    for (int xx = 0; xx < b; xx++) {
                        int y = I * b + yy, x = J * b + xx;
                        if (y >= eh || x >= ew || st[y * ew + x] != ST_PENDING) continue;
                        double g = gbuf[(size_t)q * b * b + yy * b + xx];
                        if (gstat[q] == 1) { st[y * ew + x] = ST_DONE; val[y * ew + x] = g; }
                        int gx = ex + x, gy = ey + y;
                        if (gx >= cx && gx < cx + cw && gy >= cy && gy < cy + ch) {
                            double c = g < 0 ? 0 : (g > 255 ? 255 : g);
                            out[(int64_t)gy * W + gx] = (uint8_t)rint_half_even(c);
                            if (out_g) out_g[(int64_t)gy * W + gx] = gstat[q] == 1 ? g : 0.0;
                        }
                    }
                if (gstat[q] == 2) n_empty++;
                if (rep && nrep < rep_cap) {
                    rep[nrep].tile = t; rep[nrep].I = I; rep[nrep].J = J;
                    rep[nrep].status = gstat[q]; rep[nrep].W0 = gw0[q];
                    if (useq && K > 0) memcpy(useq + (size_t)nrep * K, gseq + (size_t)q * K, sizeof(int32_t) * K);
                    nrep++;
                }
            }
            n_proc += ng;
            free(gbuf); free(gstat); free(gw0); free(gseq);
            g0 = g1;
        }
        free(val); free(st); free(bl);
    }
    free(wiso);
    free(tiles);
    if (n_rep) *n_rep = nrep;
    if (stats) { stats[0] = n_proc; stats[1] = n_empty; stats[2] = nt; stats[3] = n_core_lost; }
    return OR_OK;
}

/*
 * One block of one extended tile computed alone, with every lost pixel of the
 * tile still pending (no earlier reconstruction in its support).  Under the
 * PHASED order this is exactly what a phase-0 block sees, so sampled outputs of
 * a full-size run can be checked block by block.
 *   (ex, ey, ew, eh): the extended tile;  (I, J): the block in its grid.
 *   g[b*b]: model values at the block's pixels (row-major, unrounded).
 * Returns W0 (0: empty support, g set to 0).
 */
double oracle_fse_block_alone(const uint8_t *img, const uint8_t *mask, int32_t W, int32_t H,
                              int32_t ex, int32_t ey, int32_t ew, int32_t eh, int32_t b, int32_t B,
                              int32_t F, int32_t K, double rho, double gamma, double tau,
                              int32_t I, int32_t J, double *g) {
    (void)H;
    const int S = b + 2 * B;
    double *w = malloc(sizeof(double) * S * S), *r = malloc(sizeof(double) * S * S);
    double *cre = malloc(sizeof(double) * F * F), *cim = malloc(sizeof(double) * F * F);
    const double mc = B + (b - 1) / 2.0;
    for (int m = 0; m < S; m++)
        for (int n = 0; n < S; n++) {
            int y = I * b - B + m, x = J * b - B + n;
            double wv = 0, rv = 0;
            if (y >= 0 && y < eh && x >= 0 && x < ew) {
                int64_t gi = (int64_t)(ey + y) * W + (ex + x);
                if (!mask[gi]) {
                    wv = pow(rho, sqrt((m - mc) * (m - mc) + (n - mc) * (n - mc)));
                    rv = (double)img[gi];
                }
            }
            w[m * S + n] = wv;
            r[m * S + n] = rv;
        }
    double W0 = oracle_fse_fit(w, r, NULL, S, F, K, gamma, tau, NULL, cre, cim, NULL, NULL, NULL);
    for (int yy = 0; yy < b; yy++)
        for (int xx = 0; xx < b; xx++)
            g[yy * b + xx] = W0 > 0 ? oracle_fse_model(cre, cim, F, B + yy, B + xx) : 0.0;
    free(w); free(r); free(cre); free(cim);
    return W0;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
