/*
 * pxst_oracle.c -- plain FP64 CPU oracle for the PXST hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path calls this file: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes (Morgan et al., "speckle-tracking: a software suite for
 * ptychographic X-ray speckle tracking"):
 *   - the bilinear weights of section "Sub-pixel interpolation" (2x2 matrix form) and
 *     its masked, renormalised variant (same section, the f_M / M quotient);
 *   - make_object_map, the "Make reference image" pseudo code: scatter M*W*I and
 *     M*W^2 with bilinear weights to u - Delta_n, then divide (section "Make reference
 *     image" plus the assignment rule at the end of "Sub-pixel interpolation");
 *   - update_pixel_map, the "Update pixel mapping" pseudo code: brute-force search of
 *     error/var over an integer window centred on the current u, argmin, and the
 *     optional 3x3 paraboloid ("quadratic_refinement") for sub-pixel precision;
 *   - iterate: steps (i) and (ii) of the main loop, repeated;
 *   - calc_error, section "Calculate figures of merit": the per-pixel, per-frame error
 *     term of Eq. 1 and its sums over frames (pixel error), pixels (frame error), both
 *     (total error) and its map onto the reference plane;
 *   - update_translations, section "Update translations": the error of Eq. 1 summed over
 *     pixels for integer shifts of one frame's translation, argmin and the same 3x3
 *     paraboloid;
 *   - filter_map, the "sigma" regularisation of the pixel map (end of section "Update pixel
 *     mapping"): a Gaussian filter of the map;
 *   - update_pixel_map_frac, the first sub-pixel option of section "Update pixel mapping":
 *     the error evaluated at non-integer candidates (bilinear reads, section "Sub-pixel
 *     interpolation") instead of the paraboloid;
 *   - defocus_sweep, fit_defocus_registration of section "Initialisation": a reference
 *     image built for a range of magnifications, scored by its contrast;
 *   - integrate_map, the "integrate" option of section "Update pixel mapping": the map made
 *     irrotational by least-squares integration (conjugate gradients) and re-differentiation.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1  the bilinear weight multiplies both the M*W*I term and the M*W^2 term;
 *   R2  scatter corners outside [0,Ry) x [0,Rx) are dropped from both sums;
 *   R3  I_ref = 0 where the accumulated weight w is exactly 0 (uncovered);
 *   R4  the doubled brackets "]]" in the pseudo code are typos;
 *   R5  window centre = (floor(u0 + 1/2), floor(u1 + 1/2)); candidates are
 *       centre + (a, b), a in [-Sy, Sy], b in [-Sx, Sx];
 *   R6  I_ref is read at c - Delta_n by the masked renormalised bilinear gather with
 *       mask V = (inside the grid) and (w > 0); if the weights of the valid corners sum
 *       to zero, frame n does not enter error or var for that candidate;
 *   R7  zero valid frames => e = +inf; var == 0 => e = error (not divided);
 *   R8  argmin = first minimum in row-major window order (a outer, b inner), strict <;
 *       if every candidate is +inf the pixel keeps its u;
 *   R9  pixels with M = 0 keep their u (error and var would both be 0);
 *   R10 the paraboloid is the least-squares fit of c0 + c1 a + c2 b + c3 a^2 + c4 ab
 *       + c5 b^2 to the 3x3 errors about the argmin; if a neighbour is missing (window
 *       edge or +inf) or the Hessian is not positive definite, each axis is fitted alone
 *       by a 3-point parabola (0 shift if a point is missing or the curvature is <= 0);
 *       a shift larger than 1 on an axis is set to 0 on that axis.
 *   R11 figures of merit: eps[n,x] = (I_n(x) - W(x) R_n)^2 / var(x), R_n read at
 *       u(x) - Delta_n by the gather of R6 (u fractional); var(x) = sum over the frames
 *       valid at x of (I_n(x) - W(x))^2 (Eq. 1's sigma^2 read as in R5-R7, at the pixel's
 *       own map); frames invalid at x add nothing; var == 0 => eps = the squared residual;
 *       M = 0 pixels add nothing and their pixel error is NaN. Pixel error = sum over n,
 *       frame error = sum over x, total = sum over both.
 *   R12 reference-plane error: eps[n,x] scattered to u(x) - Delta_n with the bilinear
 *       weights of make_object_map (corners off the grid dropped), divided by the sum of
 *       the weights that landed; 0 where none did.
 *   R13 update_translations: candidates Delta_n + (a, b), a in [-Ty, Ty], b in [-Tx, Tx]
 *       (integer shifts of the image); e_n(a, b) = the mean, over the pixels with M = 1,
 *       var(x) > 0 (var of R11 with the current translations) and a valid read at
 *       u(x) - Delta_n - (a, b), of (I_n(x) - W(x) R)^2 / var(x) (a mean, not a sum, so
 *       that shifting pixels off the reference is not rewarded); +inf with no such pixel;
 *       argmin as R8, the fit as R10; Delta_n <- Delta_n + (a*, b*) + fit.
 *   R17 integrate: the least-squares projection of the map onto discrete gradient fields
 *       over the good pixels (central differences where both neighbours along an axis are
 *       good, second-order one-sided ones where two on one side are, first-order where
 *       only one is), solved by conjugate gradients on the normal equations; see
 *       pxst_oracle_integrate_map.
 *
 * Array conventions: frames float32 [N][ny][nx]; W float32 [ny][nx]; M uint8 [ny][nx];
 * u float64 [2][ny][nx] (u[0] rows, u[1] columns, reference-pixel units);
 * delta float64 [N][2]; Iref, w float64 [Ry][Rx].
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math, no fused
 * multiply-add, so the x86 and Arm builds round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------- */
/* bilinear weights (section "Sub-pixel interpolation")                               */
/* ---------------------------------------------------------------------------------- */

/* For the point (a, b): i0 = floor(a), j0 = floor(b), x = a - i0, y = b - j0.
 * f(a,b) ~ [1-x, x] . [[f00, f01], [f10, f11]] . [1-y, y]^T, so corner (di, dj)
 * carries weight (di ? x : 1-x) * (dj ? y : 1-y). Order: 00, 01, 10, 11. */
void pxst_oracle_bilinear(double a, double b, int64_t *i0, int64_t *j0, double wt[4])
{
    double fi = floor(a), fj = floor(b);
    double x = a - fi, y = b - fj;
    *i0 = (int64_t)fi;
    *j0 = (int64_t)fj;
    wt[0] = (1.0 - x) * (1.0 - y);
    wt[1] = (1.0 - x) * y;
    wt[2] = x * (1.0 - y);
    wt[3] = x * y;
}

/* Masked, renormalised gather: sum_k wt_k V_k f_k / sum_k wt_k V_k, with
 * V = inside the grid and w > 0 (reading R6). Returns 1 and stores the value if the
 * valid weights sum to more than zero, else returns 0 (frame invalid). */
int pxst_oracle_gather(const double *Iref, const double *w, int64_t Ry, int64_t Rx,
                       double q0, double q1, double *out)
{
    int64_t i0, j0;
    double wt[4];
    pxst_oracle_bilinear(q0, q1, &i0, &j0, wt);
    double num = 0.0, den = 0.0;
    for (int k = 0; k < 4; ++k) {
        int64_t ii = i0 + (k >> 1), jj = j0 + (k & 1);
        if (wt[k] == 0.0) continue;                 /* contributes nothing either way */
        if (ii < 0 || ii >= Ry || jj < 0 || jj >= Rx) continue;
        double wc = w[ii * Rx + jj];
        if (!(wc > 0.0)) continue;
        num += wt[k] * Iref[ii * Rx + jj];
        den += wt[k];
    }
    if (!(den > 0.0)) return 0;
    *out = num / den;
    return 1;
}

/* ---------------------------------------------------------------------------------- */
/* make_object_map (section "Make reference image")                                  */
/* ---------------------------------------------------------------------------------- */

void pxst_oracle_make_object_map(int N, int ny, int nx, int Ry, int Rx,
                                 const float *frames, const float *W, const uint8_t *M,
                                 const double *u, const double *delta,
                                 double *Iref, double *w)
{
    const int64_t P = (int64_t)ny * nx, R = (int64_t)Ry * Rx;
    memset(Iref, 0, sizeof(double) * R);
    memset(w, 0, sizeof(double) * R);
    for (int n = 0; n < N; ++n) {
        for (int i = 0; i < ny; ++i) {
            for (int j = 0; j < nx; ++j) {
                const int64_t p = (int64_t)i * nx + j;
                /* M is 0 or 1: for M = 0 both added terms are exactly 0 */
                if (!M[p]) continue;
                const double m = 1.0;
                const double Wv = (double)W[p];
                const double I = (double)frames[(int64_t)n * P + p];
                const double a = u[p] - delta[2 * n + 0];
                const double b = u[P + p] - delta[2 * n + 1];
                int64_t i0, j0;
                double wt[4];
                pxst_oracle_bilinear(a, b, &i0, &j0, wt);
                for (int k = 0; k < 4; ++k) {
                    int64_t ii = i0 + (k >> 1), jj = j0 + (k & 1);
                    if (ii < 0 || ii >= Ry || jj < 0 || jj >= Rx) continue;   /* R2 */
                    Iref[ii * Rx + jj] += wt[k] * m * Wv * I;                  /* R1 */
                    w[ii * Rx + jj] += wt[k] * m * Wv * Wv;
                }
            }
        }
    }
    for (int64_t c = 0; c < R; ++c)                                            /* R3 */
        Iref[c] = (w[c] > 0.0) ? Iref[c] / w[c] : 0.0;
}

/* ---------------------------------------------------------------------------------- */
/* quadratic refinement (end of section "Update pixel mapping")                      */
/* ---------------------------------------------------------------------------------- */

static int finite_(double v) { return isfinite(v); }

/* f[9]: normalised errors at (da, db) in {-1,0,1}^2, da outer, db inner; +inf marks
 * a missing neighbour. Returns the sub-pixel shift (da, db) of the minimum (R10). */
void pxst_oracle_quadratic_fit(const double f[9], double *da_out, double *db_out)
{
    double da = 0.0, db = 0.0;
    int complete = 1;
    for (int k = 0; k < 9; ++k) complete &= finite_(f[k]);
    int done = 0;
    if (complete) {
        double s = 0, sa = 0, sb = 0, sab = 0, a2 = 0, b2 = 0;
        for (int ia = -1; ia <= 1; ++ia)
            for (int ib = -1; ib <= 1; ++ib) {
                double v = f[(ia + 1) * 3 + (ib + 1)];
                s += v;
                sa += ia * v;
                sb += ib * v;
                sab += ia * ib * v;
                if (ia != 0) a2 += v;
                if (ib != 0) b2 += v;
            }
        double c1 = sa / 6.0, c2 = sb / 6.0, c4 = sab / 4.0;
        double c3 = (a2 - 2.0 * (s - a2)) / 6.0;
        double c5 = (b2 - 2.0 * (s - b2)) / 6.0;
        double det = 4.0 * c3 * c5 - c4 * c4;
        if (c3 > 0.0 && det > 0.0) {
            /* [2c3 c4; c4 2c5] (da, db)^T = -(c1, c2)^T */
            da = (-2.0 * c5 * c1 + c4 * c2) / det;
            db = (-2.0 * c3 * c2 + c4 * c1) / det;
            done = 1;
        }
    }
    if (!done) {
        double fm = f[1], f0 = f[4], fp = f[7];           /* along a, db = 0 */
        da = 0.0;
        if (finite_(fm) && finite_(fp) && finite_(f0)) {
            double k = fm - 2.0 * f0 + fp;
            if (k > 0.0) da = (fm - fp) / (2.0 * k);
        }
        fm = f[3]; fp = f[5];                             /* along b, da = 0 */
        db = 0.0;
        if (finite_(fm) && finite_(fp) && finite_(f0)) {
            double k = fm - 2.0 * f0 + fp;
            if (k > 0.0) db = (fm - fp) / (2.0 * k);
        }
    }
    if (!(fabs(da) <= 1.0)) da = 0.0;
    if (!(fabs(db) <= 1.0)) db = 0.0;
    *da_out = da;
    *db_out = db;
}

/* ---------------------------------------------------------------------------------- */
/* update_pixel_map (section "Update pixel mapping")                                 */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    int N, ny, nx, Ry, Rx, Sy, Sx;
    const float *frames, *W;
    const uint8_t *M;
    const double *Iref, *w, *delta, *u;
} upm_ctx;

/* The whole error window of pixel p: e[(a+Sy)*(2Sx+1) + (b+Sx)] (R5-R7). */
static void pixel_window(const upm_ctx *c, int64_t p, double *e, int64_t *ci, int64_t *cj)
{
    const int64_t P = (int64_t)c->ny * c->nx;
    const int wx = 2 * c->Sx + 1;
    *ci = (int64_t)floor(c->u[p] + 0.5);
    *cj = (int64_t)floor(c->u[P + p] + 0.5);
    const double Wv = (double)c->W[p];
    for (int a = -c->Sy; a <= c->Sy; ++a) {
        for (int b = -c->Sx; b <= c->Sx; ++b) {
            double error = 0.0, var = 0.0;
            int nvalid = 0;
            for (int n = 0; n < c->N; ++n) {
                double R;
                double q0 = (double)(*ci + a) - c->delta[2 * n + 0];
                double q1 = (double)(*cj + b) - c->delta[2 * n + 1];
                if (!pxst_oracle_gather(c->Iref, c->w, c->Ry, c->Rx, q0, q1, &R)) continue;
                const double I = (double)c->frames[(int64_t)n * P + p];
                const double d = I - Wv * R;
                const double v = I - Wv;
                error += d * d;
                var += v * v;
                nvalid += 1;
            }
            double ev;
            if (nvalid == 0) ev = INFINITY;
            else if (var > 0.0) ev = error / var;
            else ev = error;
            e[(a + c->Sy) * wx + (b + c->Sx)] = ev;
        }
    }
}

/* Search + argmin + optional fit for one pixel; writes u_out[0..1] and *err. */
static void update_one(const upm_ctx *c, int quadratic, int64_t p, double *e,
                       double *u0_out, double *u1_out, double *err)
{
    const int64_t P = (int64_t)c->ny * c->nx;
    if (!c->M[p]) {                                          /* R9 */
        *u0_out = c->u[p];
        *u1_out = c->u[P + p];
        *err = NAN;
        return;
    }
    int64_t ci, cj;
    pixel_window(c, p, e, &ci, &cj);
    const int wy = 2 * c->Sy + 1, wx = 2 * c->Sx + 1;
    int best = 0;
    for (int k = 1; k < wy * wx; ++k)                          /* R8 */
        if (e[k] < e[best]) best = k;
    if (!(e[best] < INFINITY)) {
        *u0_out = c->u[p];
        *u1_out = c->u[P + p];
        *err = INFINITY;
        return;
    }
    const int ia = best / wx, ib = best % wx;
    double da = 0.0, db = 0.0;
    if (quadratic) {
        double f[9];
        for (int sa = -1; sa <= 1; ++sa)
            for (int sb = -1; sb <= 1; ++sb) {
                int na = ia + sa, nb = ib + sb;
                f[(sa + 1) * 3 + (sb + 1)] =
                    (na < 0 || na >= wy || nb < 0 || nb >= wx) ? INFINITY : e[na * wx + nb];
            }
        pxst_oracle_quadratic_fit(f, &da, &db);
    }
    *u0_out = (double)(ci + ia - c->Sy) + da;
    *u1_out = (double)(cj + ib - c->Sx) + db;
    *err = e[best];
}

/* Error window of one pixel (for tests): e has (2Sy+1)(2Sx+1) entries. */
void pxst_oracle_pixel_window(int N, int ny, int nx, int Ry, int Rx, int Sy, int Sx,
                              const float *frames, const float *W, const uint8_t *M,
                              const double *Iref, const double *w, const double *delta,
                              const double *u, int64_t p, double *e, int64_t *centre)
{
    upm_ctx c = {N, ny, nx, Ry, Rx, Sy, Sx, frames, W, M, Iref, w, delta, u};
    pixel_window(&c, p, e, &centre[0], &centre[1]);
}

/* update_pixel_map over rows [row0, row1); u is read from u_in and written to u_out
 * (they may alias: each pixel reads only its own entries). err_out may be NULL. */
void pxst_oracle_update_pixel_map(int N, int ny, int nx, int Ry, int Rx, int Sy, int Sx,
                                  int quadratic, const float *frames, const float *W,
                                  const uint8_t *M, const double *Iref, const double *w,
                                  const double *delta, const double *u_in, double *u_out,
                                  double *err_out, int row0, int row1, int nthreads)
{
    upm_ctx c = {N, ny, nx, Ry, Rx, Sy, Sx, frames, W, M, Iref, w, delta, u_in};
    const int64_t P = (int64_t)ny * nx;
    const int nwin = (2 * Sy + 1) * (2 * Sx + 1);
    if (nthreads <= 0) nthreads = 1;
    #pragma omp parallel num_threads(nthreads)
    {
        double *e = (double *)malloc(sizeof(double) * nwin);
        #pragma omp for schedule(dynamic, 1)
        for (int i = row0; i < row1; ++i) {
            for (int j = 0; j < nx; ++j) {
                const int64_t p = (int64_t)i * nx + j;
                double u0, u1, er;
                update_one(&c, quadratic, p, e, &u0, &u1, &er);
                u_out[p] = u0;
                u_out[P + p] = u1;
                if (err_out) err_out[p] = er;
            }
        }
        free(e);
    }
}

/* The same update for an arbitrary list of pixels (sampled parity at full size):
 * writes u_out[2*k+0..1] and err_out[k] for pixel pix[k]. */
void pxst_oracle_update_pixels(int N, int ny, int nx, int Ry, int Rx, int Sy, int Sx,
                               int quadratic, const float *frames, const float *W,
                               const uint8_t *M, const double *Iref, const double *w,
                               const double *delta, const double *u, const int64_t *pix,
                               int64_t npix, double *u_out, double *err_out, int nthreads)
{
    upm_ctx c = {N, ny, nx, Ry, Rx, Sy, Sx, frames, W, M, Iref, w, delta, u};
    const int nwin = (2 * Sy + 1) * (2 * Sx + 1);
    if (nthreads <= 0) nthreads = 1;
    #pragma omp parallel num_threads(nthreads)
    {
        double *e = (double *)malloc(sizeof(double) * nwin);
        #pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < npix; ++k)
            update_one(&c, quadratic, pix[k], e, &u_out[2 * k], &u_out[2 * k + 1], &err_out[k]);
        free(e);
    }
}

/* ---------------------------------------------------------------------------------- */
/* reference terms: expanding the square of the update step's error,                  */
/* sum_n V (I - W R)^2 = sum_n V I^2 - 2 W sum_n V I R + W^2 sum_n V R^2, the last sum */
/* depends on the candidate c only.                                                   */
/* ---------------------------------------------------------------------------------- */

/* T[c] = sum_n V_n(c) R_n(c)^2 and nvalid[c] = sum_n V_n(c) for every reference pixel
 * c, with R_n(c) the masked renormalised read of I_ref at c - Delta_n (reading R6). */
void pxst_oracle_reference_terms(int N, int Ry, int Rx, const double *Iref, const double *w,
                                 const double *delta, double *T, int32_t *nvalid, int nthreads)
{
    if (nthreads <= 0) nthreads = 1;
    #pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int cy = 0; cy < Ry; ++cy) {
        for (int cx = 0; cx < Rx; ++cx) {
            double t = 0.0;
            int nv = 0;
            for (int n = 0; n < N; ++n) {
                double R;
                if (!pxst_oracle_gather(Iref, w, Ry, Rx, (double)cy - delta[2 * n + 0],
                                        (double)cx - delta[2 * n + 1], &R))
                    continue;
                t += R * R;
                nv += 1;
            }
            T[(int64_t)cy * Rx + cx] = t;
            nvalid[(int64_t)cy * Rx + cx] = nv;
        }
    }
}

/* ---------------------------------------------------------------------------------- */
/* iterate: main loop steps (i) and (ii)                                              */
/* ---------------------------------------------------------------------------------- */

void pxst_oracle_iterate(int N, int ny, int nx, int Ry, int Rx, int Sy, int Sx, int quadratic,
                         int n_iter, const float *frames, const float *W, const uint8_t *M,
                         const double *delta, double *u_inout, double *Iref, double *w,
                         double *err_out, int nthreads)
{
    for (int it = 0; it < n_iter; ++it) {
        pxst_oracle_make_object_map(N, ny, nx, Ry, Rx, frames, W, M, u_inout, delta, Iref, w);
        pxst_oracle_update_pixel_map(N, ny, nx, Ry, Rx, Sy, Sx, quadratic, frames, W, M, Iref,
                                     w, delta, u_inout, u_inout, err_out, 0, ny, nthreads);
    }
    /* I_ref and w are those built in the last iteration's step (i) */
}

/* ---------------------------------------------------------------------------------- */
/* defocus registration (fit_defocus_registration, section "Initialisation")          */
/* ---------------------------------------------------------------------------------- */

/* R16 a magnification guess M scales the map about the detector's central pixel
 *     (i_c, j_c) = (ny/2, nx/2) (integer division): u'_a(x) = u_a(x_c) + s_a (u_a(x) - u_a(x_c))
 *     per axis a, s_a the ratio of the guessed to the current magnification, the translations
 *     unchanged; the reference image is make_object_map with u'; its contrast is the standard
 *     deviation over its mean, both over the reference pixels with w > 0 (0 if none or the
 *     mean is 0). contrast[ky * nsx + kx] for the pair (sy[ky], sx[kx]). */
double pxst_oracle_contrast(int64_t R, const double *Iref, const double *w)
{
    double s1 = 0.0, s2 = 0.0;
    int64_t n = 0;
    for (int64_t c = 0; c < R; ++c) {
        if (!(w[c] > 0.0)) continue;
        s1 += Iref[c];
        n += 1;
    }
    if (n == 0) return 0.0;
    const double mean = s1 / (double)n;
    for (int64_t c = 0; c < R; ++c) {
        if (!(w[c] > 0.0)) continue;
        const double d = Iref[c] - mean;
        s2 += d * d;
    }
    if (mean == 0.0) return 0.0;
    return sqrt(s2 / (double)n) / mean;
}

void pxst_oracle_defocus_sweep(int N, int ny, int nx, int Ry, int Rx, const float *frames, const float *W,
                               const uint8_t *M, const double *u, const double *delta, int nsy, const double *sy,
                               int nsx, const double *sx, double *contrast)
{
    const int64_t P = (int64_t)ny * nx, R = (int64_t)Ry * Rx;
    const int64_t pc = (int64_t)(ny / 2) * nx + nx / 2;
    double *us = (double *)malloc(sizeof(double) * 2 * (size_t)P);
    double *Iref = (double *)malloc(sizeof(double) * (size_t)R);
    double *w = (double *)malloc(sizeof(double) * (size_t)R);
    for (int ky = 0; ky < nsy; ++ky) {
        for (int kx = 0; kx < nsx; ++kx) {
            for (int64_t p = 0; p < P; ++p) {
                us[p] = u[pc] + sy[ky] * (u[p] - u[pc]);
                us[P + p] = u[P + pc] + sx[kx] * (u[P + p] - u[P + pc]);
            }
            pxst_oracle_make_object_map(N, ny, nx, Ry, Rx, frames, W, M, us, delta, Iref, w);
            contrast[ky * nsx + kx] = pxst_oracle_contrast(R, Iref, w);
        }
    }
    free(us);
    free(Iref);
    free(w);
}

/* ---------------------------------------------------------------------------------- */
/* fractional candidates (the non-integer option of section "Update pixel mapping")   */
/* ---------------------------------------------------------------------------------- */

/* R15 after the integer search (R5-R8, no fit) of pixel p gives c*, the candidates
 *     c* + (a, b) / s, a, b in [-s, s], are evaluated by the same rule (R6, R7) with
 *     fractional reads; u = the first minimum in row-major order (a outer), its error is
 *     reported; a pixel whose integer search found no finite error keeps its u. */
void pxst_oracle_update_pixel_map_frac(int N, int ny, int nx, int Ry, int Rx, int Sy, int Sx, int sub,
                                       const float *frames, const float *W, const uint8_t *M,
                                       const double *Iref, const double *w, const double *delta,
                                       const double *u_in, double *u_out, double *err_out, int nthreads)
{
    upm_ctx c = {N, ny, nx, Ry, Rx, Sy, Sx, frames, W, M, Iref, w, delta, u_in};
    const int64_t P = (int64_t)ny * nx;
    const int nwin = (2 * Sy + 1) * (2 * Sx + 1);
    if (nthreads <= 0) nthreads = 1;
    #pragma omp parallel num_threads(nthreads)
    {
        double *e = (double *)malloc(sizeof(double) * nwin);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < P; ++p) {
            double u0, u1, er;
            update_one(&c, 0, p, e, &u0, &u1, &er);
            if (M[p] && er < INFINITY) {
                const double Wv = (double)W[p];
                double best_e = INFINITY, b0 = u0, b1 = u1;
                for (int a = -sub; a <= sub; ++a) {
                    for (int b = -sub; b <= sub; ++b) {
                        const double c0 = u0 + (double)a / sub, c1 = u1 + (double)b / sub;
                        double error = 0.0, var = 0.0;
                        int nvalid = 0;
                        for (int n = 0; n < N; ++n) {
                            double R;
                            if (!pxst_oracle_gather(Iref, w, Ry, Rx, c0 - delta[2 * n], c1 - delta[2 * n + 1], &R))
                                continue;
                            const double In = (double)frames[(int64_t)n * P + p];
                            const double res = In - Wv * R, dev = In - Wv;
                            error += res * res;
                            var += dev * dev;
                            nvalid += 1;
                        }
                        const double ev = nvalid == 0 ? INFINITY : (var > 0.0 ? error / var : error);
                        if (ev < best_e) {                                  /* strict <: first minimum */
                            best_e = ev;
                            b0 = c0;
                            b1 = c1;
                        }
                    }
                }
                u0 = b0;
                u1 = b1;
                er = best_e;
            }
            u_out[p] = u0;
            u_out[P + p] = u1;
            if (err_out) err_out[p] = er;
        }
        free(e);
    }
}

/* ---------------------------------------------------------------------------------- */
/* the irrotational constraint (the "integrate" option of the update)                 */
/* ---------------------------------------------------------------------------------- */

/* R17 u is the gradient of a scalar (u = x - lambda z / (2 pi) grad Phi, section "Update
 *     pixel mapping"): the map is integrated by least squares and differentiated again.
 *     Equations, one per good pixel p and axis a (e = the unit step along a), each the
 *     derivative of Psi at p along a set equal to u_a[p], by the first of these stencils
 *     whose pixels are all good:
 *        central          (Psi[p+e] - Psi[p-e]) / 2
 *        forward, 2nd ord (-3 Psi[p] + 4 Psi[p+e] - Psi[p+2e]) / 2
 *        backward, 2nd ord (3 Psi[p] - 4 Psi[p-e] + Psi[p-2e]) / 2
 *        forward          Psi[p+e] - Psi[p]
 *        backward         Psi[p] - Psi[p-e]
 *     (none if p has no good neighbour along a). Psi on the good pixels minimises the sum of
 *     squared residuals, by conjugate gradients on the normal equations G^T G Psi = G^T u
 *     from Psi = 0, until |G^T (u - G Psi)| <= tol |G^T u| or max_iter steps; the output is
 *     u_a[p] = (G Psi) of each equation (a pixel and axis with no equation, and every M = 0
 *     pixel, keep u). Every stencil but the last two is exact for a quadratic Psi. Returns
 *     the steps taken; *resid gets the final relative residual. */

/* the stencil of pixel (i, j) on axis a: n taps at offsets off[k] (in steps along a) with
 * coefficients c[k]; n = 0: no equation */
static int integ_stencil(int ny, int nx, const uint8_t *M, int i, int j, int a, int off[3], double c[3]) {
    if (!M[(size_t)i * nx + j]) return 0;
    const int len = a == 0 ? ny : nx, pos = a == 0 ? i : j;
#define GOOD(k) (pos + (k) >= 0 && pos + (k) < len && M[(size_t)(a == 0 ? i + (k) : i) * nx + (a == 0 ? j : j + (k))])
    if (GOOD(1) && GOOD(-1)) { off[0] = 1; c[0] = 0.5; off[1] = -1; c[1] = -0.5; return 2; }
    if (GOOD(1) && GOOD(2)) { off[0] = 0; c[0] = -1.5; off[1] = 1; c[1] = 2.0; off[2] = 2; c[2] = -0.5; return 3; }
    if (GOOD(-1) && GOOD(-2)) { off[0] = 0; c[0] = 1.5; off[1] = -1; c[1] = -2.0; off[2] = -2; c[2] = 0.5; return 3; }
    if (GOOD(1)) { off[0] = 1; c[0] = 1.0; off[1] = 0; c[1] = -1.0; return 2; }
    if (GOOD(-1)) { off[0] = 0; c[0] = 1.0; off[1] = -1; c[1] = -1.0; return 2; }
#undef GOOD
    return 0;
}

/* g = G psi: one value per pixel and axis (0 where there is no equation) */
static void integ_apply_G(int ny, int nx, const uint8_t *M, const double *psi, double *g) {
    const size_t P = (size_t)ny * nx;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                const size_t p = (size_t)i * nx + j;
                const long step = a == 0 ? nx : 1;
                int off[3];
                double c[3];
                const int n = integ_stencil(ny, nx, M, i, j, a, off, c);
                double v = 0.0;
                for (int k = 0; k < n; ++k) v += c[k] * psi[(long)p + off[k] * step];
                g[a * P + p] = v;
            }
}

/* y = G^T g: every equation adds its coefficients times its value to the pixels it reads */
static void integ_apply_GT(int ny, int nx, const uint8_t *M, const double *g, double *y) {
    const size_t P = (size_t)ny * nx;
    for (size_t p = 0; p < P; ++p) y[p] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                const size_t p = (size_t)i * nx + j;
                const long step = a == 0 ? nx : 1;
                int off[3];
                double c[3];
                const int n = integ_stencil(ny, nx, M, i, j, a, off, c);
                for (int k = 0; k < n; ++k) y[(long)p + off[k] * step] += c[k] * g[a * P + p];
            }
}

static double integ_dot(size_t n, const double *x, const double *y) {
    double s = 0.0;
    for (size_t k = 0; k < n; ++k) s += x[k] * y[k];
    return s;
}

int pxst_oracle_integrate_map(int ny, int nx, const uint8_t *M, const double *u_in, int max_iter, double tol,
                              double *u_out, double *resid) {
    const size_t P = (size_t)ny * nx;
    double *psi = calloc(P, sizeof(double)), *r = calloc(P, sizeof(double)), *d = calloc(P, sizeof(double));
    double *q = calloc(P, sizeof(double)), *g = calloc(2 * P, sizeof(double)), *b = calloc(P, sizeof(double));
    double *ue = calloc(2 * P, sizeof(double));
    /* the data of each equation (0 where there is none) */
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                const size_t p = (size_t)i * nx + j;
                int off[3];
                double c[3];
                ue[a * P + p] = integ_stencil(ny, nx, M, i, j, a, off, c) ? u_in[a * P + p] : 0.0;
            }
    integ_apply_GT(ny, nx, M, ue, b);                      /* b = G^T u */
    for (size_t p = 0; p < P; ++p) { r[p] = b[p]; d[p] = b[p]; }
    const double bb = integ_dot(P, b, b);
    double rr = bb;
    int it = 0;
    while (it < max_iter && rr > tol * tol * bb && bb > 0.0) {
        integ_apply_G(ny, nx, M, d, g);                    /* q = G^T G d */
        integ_apply_GT(ny, nx, M, g, q);
        const double dq = integ_dot(P, d, q);
        if (!(dq > 0.0)) break;
        const double alpha = rr / dq;
        for (size_t p = 0; p < P; ++p) {
            psi[p] += alpha * d[p];
            r[p] -= alpha * q[p];
        }
        const double rr_new = integ_dot(P, r, r);
        const double beta = rr_new / rr;
        for (size_t p = 0; p < P; ++p) d[p] = r[p] + beta * d[p];
        rr = rr_new;
        ++it;
    }
    if (resid) *resid = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    integ_apply_G(ny, nx, M, psi, g);
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                const size_t p = (size_t)i * nx + j;
                int off[3];
                double c[3];
                u_out[a * P + p] = integ_stencil(ny, nx, M, i, j, a, off, c) ? g[a * P + p] : u_in[a * P + p];
            }
    free(psi); free(r); free(d); free(q); free(g); free(b); free(ue);
    return it;
}

/* ---------------------------------------------------------------------------------- */
/* regularisation of the pixel map (the "sigma" option of the update)                 */
/* ---------------------------------------------------------------------------------- */

/* R14 u_f(x) = sum_y g(x - y) M(y) u(y) / sum_y g(x - y) M(y) for M(x) = 1, with
 *     g(d) = exp(-|d|^2 / (2 sigma^2)) for |d_i|, |d_j| <= r = floor(4 sigma + 1/2) (a square
 *     support, so the 2-D kernel is the product of two 1-D ones); M = 0 pixels keep u;
 *     sigma <= 0 leaves u unchanged. Direct 2-D sum per pixel. */
void pxst_oracle_filter_map(int ny, int nx, double sigma, const uint8_t *M, const double *u_in, double *u_out)
{
    const int64_t P = (int64_t)ny * nx;
    memcpy(u_out, u_in, sizeof(double) * 2 * (size_t)P);
    if (!(sigma > 0.0)) return;
    const int r = (int)floor(4.0 * sigma + 0.5);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < ny; ++i) {
        for (int j = 0; j < nx; ++j) {
            const int64_t p = (int64_t)i * nx + j;
            if (!M[p]) continue;
            double num0 = 0.0, num1 = 0.0, den = 0.0;
            for (int a = -r; a <= r; ++a) {
                const int ii = i + a;
                if (ii < 0 || ii >= ny) continue;
                for (int b = -r; b <= r; ++b) {
                    const int jj = j + b;
                    if (jj < 0 || jj >= nx) continue;
                    const int64_t q = (int64_t)ii * nx + jj;
                    if (!M[q]) continue;
                    const double g = exp(-(double)(a * a + b * b) / (2.0 * sigma * sigma));
                    num0 += g * u_in[q];
                    num1 += g * u_in[P + q];
                    den += g;
                }
            }
            u_out[p] = num0 / den;
            u_out[P + p] = num1 / den;
        }
    }
}

/* ---------------------------------------------------------------------------------- */
/* figures of merit (section "Calculate figures of merit")                           */
/* ---------------------------------------------------------------------------------- */

/* var(x) of R11 for pixel p at its own map with translations delta (-1 if M = 0). */
static double pixel_var(int N, int64_t P, int Ry, int Rx, const float *frames, const float *W,
                        const uint8_t *M, const double *Iref, const double *w, const double *u,
                        const double *delta, int64_t p)
{
    if (!M[p]) return -1.0;
    const double Wv = (double)W[p];
    double s2 = 0.0;
    for (int n = 0; n < N; ++n) {
        double R;
        if (!pxst_oracle_gather(Iref, w, Ry, Rx, u[p] - delta[2 * n], u[P + p] - delta[2 * n + 1], &R)) continue;
        const double v = (double)frames[(int64_t)n * P + p] - Wv;
        s2 += v * v;
    }
    return s2;
}

/* pixel_err [ny][nx], frame_err [N], *total and ref_err [Ry][Rx] (R11, R12). Serial: the
 * sums run in pixel order, frame order inside. */
void pxst_oracle_calc_error(int N, int ny, int nx, int Ry, int Rx, const float *frames, const float *W,
                            const uint8_t *M, const double *Iref, const double *w, const double *u,
                            const double *delta, double *pixel_err, double *frame_err, double *total,
                            double *ref_err)
{
    const int64_t P = (int64_t)ny * nx, R = (int64_t)Ry * Rx;
    double *num = (double *)calloc((size_t)R, sizeof(double));
    double *den = (double *)calloc((size_t)R, sizeof(double));
    for (int n = 0; n < N; ++n) frame_err[n] = 0.0;
    double tot = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        const double var = pixel_var(N, P, Ry, Rx, frames, W, M, Iref, w, u, delta, p);
        if (var < 0.0) {
            pixel_err[p] = NAN;
            continue;
        }
        const double Wv = (double)W[p];
        double pe = 0.0;
        for (int n = 0; n < N; ++n) {
            const double q0 = u[p] - delta[2 * n], q1 = u[P + p] - delta[2 * n + 1];
            double Rv;
            if (!pxst_oracle_gather(Iref, w, Ry, Rx, q0, q1, &Rv)) continue;
            const double d = (double)frames[(int64_t)n * P + p] - Wv * Rv;
            const double eps = var > 0.0 ? d * d / var : d * d;
            pe += eps;
            frame_err[n] += eps;
            int64_t i0, j0;
            double wt[4];
            pxst_oracle_bilinear(q0, q1, &i0, &j0, wt);
            for (int k = 0; k < 4; ++k) {
                const int64_t ii = i0 + (k >> 1), jj = j0 + (k & 1);
                if (ii < 0 || ii >= Ry || jj < 0 || jj >= Rx) continue;
                num[ii * Rx + jj] += wt[k] * eps;
                den[ii * Rx + jj] += wt[k];
            }
        }
        pixel_err[p] = pe;
        tot += pe;
    }
    *total = tot;
    for (int64_t c = 0; c < R; ++c) ref_err[c] = den[c] > 0.0 ? num[c] / den[c] : 0.0;
    free(num);
    free(den);
}

/* ---------------------------------------------------------------------------------- */
/* update_translations (section "Update translations")                               */
/* ---------------------------------------------------------------------------------- */

/* The error window of frame n: e[(a+Ty)*(2Tx+1) + (b+Tx)] (R13), given var[p]. */
static void frame_window(int N, int ny, int nx, int Ry, int Rx, int Ty, int Tx, const float *frames,
                         const float *W, const uint8_t *M, const double *Iref, const double *w,
                         const double *u, const double *delta, const double *var, int n, double *e)
{
    const int64_t P = (int64_t)ny * nx;
    const int wx = 2 * Tx + 1;
    (void)N;
    for (int a = -Ty; a <= Ty; ++a) {
        for (int b = -Tx; b <= Tx; ++b) {
            double sum = 0.0;
            int64_t cnt = 0;
            for (int64_t p = 0; p < P; ++p) {
                if (!M[p] || !(var[p] > 0.0)) continue;
                double Rv;
                const double q0 = u[p] - (delta[2 * n] + a), q1 = u[P + p] - (delta[2 * n + 1] + b);
                if (!pxst_oracle_gather(Iref, w, Ry, Rx, q0, q1, &Rv)) continue;
                const double d = (double)frames[(int64_t)n * P + p] - (double)W[p] * Rv;
                sum += d * d / var[p];
                cnt += 1;
            }
            e[(a + Ty) * wx + (b + Tx)] = cnt > 0 ? sum / (double)cnt : INFINITY;
        }
    }
}

/* Error window of one frame (for tests): e has (2Ty+1)(2Tx+1) entries. */
void pxst_oracle_frame_window(int N, int ny, int nx, int Ry, int Rx, int Ty, int Tx, const float *frames,
                              const float *W, const uint8_t *M, const double *Iref, const double *w,
                              const double *u, const double *delta, int n, double *e)
{
    const int64_t P = (int64_t)ny * nx;
    double *var = (double *)malloc(sizeof(double) * (size_t)P);
    for (int64_t p = 0; p < P; ++p) var[p] = pixel_var(N, P, Ry, Rx, frames, W, M, Iref, w, u, delta, p);
    frame_window(N, ny, nx, Ry, Rx, Ty, Tx, frames, W, M, Iref, w, u, delta, var, n, e);
    free(var);
}

/* New translations delta_out [N][2] and each frame's error at its argmin err_out [N]. */
void pxst_oracle_update_translations(int N, int ny, int nx, int Ry, int Rx, int Ty, int Tx, int quadratic,
                                     const float *frames, const float *W, const uint8_t *M, const double *Iref,
                                     const double *w, const double *u, const double *delta_in,
                                     double *delta_out, double *err_out)
{
    const int64_t P = (int64_t)ny * nx;
    const int wy = 2 * Ty + 1, wx = 2 * Tx + 1;
    double *var = (double *)malloc(sizeof(double) * (size_t)P);
    for (int64_t p = 0; p < P; ++p) var[p] = pixel_var(N, P, Ry, Rx, frames, W, M, Iref, w, u, delta_in, p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < N; ++n) {
        double *e = (double *)malloc(sizeof(double) * (size_t)(wy * wx));
        frame_window(N, ny, nx, Ry, Rx, Ty, Tx, frames, W, M, Iref, w, u, delta_in, var, n, e);
        int best = -1;
        double be = INFINITY;
        for (int k = 0; k < wy * wx; ++k)
            if (e[k] < be) {                                  /* R8: strict <, first minimum */
                be = e[k];
                best = k;
            }
        delta_out[2 * n] = delta_in[2 * n];
        delta_out[2 * n + 1] = delta_in[2 * n + 1];
        err_out[n] = be;
        if (best >= 0) {
            const int ia = best / wx, ib = best % wx;
            double da = 0.0, db = 0.0;
            if (quadratic) {
                double f[9];
                for (int q = 0; q < 9; ++q) {
                    const int a2 = ia + q / 3 - 1, b2 = ib + q % 3 - 1;
                    f[q] = (a2 < 0 || a2 >= wy || b2 < 0 || b2 >= wx) ? INFINITY : e[a2 * wx + b2];
                }
                pxst_oracle_quadratic_fit(f, &da, &db);
            }
            delta_out[2 * n] = delta_in[2 * n] + (double)(ia - Ty) + da;
            delta_out[2 * n + 1] = delta_in[2 * n + 1] + (double)(ib - Tx) + db;
        }
        free(e);
    }
    free(var);
}
