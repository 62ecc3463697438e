/*
 * FP64 CPU oracle for the DIA kernel fit (PyTorchDIA, arXiv 2104.13715).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no header, constant or helper with the CUDA
 * path: every definition below is written out again from the paper.
 *
 * What it computes, by direct nested loops in double precision:
 *
 *   model image     M_ij = sum_{l,m} K_lm R_(i+l)(j+m) + B_ij         (Sec. 2.1, Eq. 2)
 *                   with centred offsets l,m in [-h, h], kernel side 2h+1,
 *                   defined only where the whole kernel footprint lies
 *                   inside R, i.e. i,j in [h, N-h)                     (Sec. 2.1, N_data)
 *   background      B_ij = B0 (degree 0), or the polynomial of degree d
 *                   B = sum_{p=0..d} sum_{q=0..d-p} b_pq eta^p xi^q     (Sec. 2.6, Eq. 18)
 *                   eta = (j - x_c)/N_x, xi = (i - y_c)/N_y            (Sec. 2.6, Eq. 19)
 *                   with x = column j, y = row i of the full image,
 *                   x_c = (W-1)/2, y_c = (H-1)/2, N_x = W, N_y = H
 *   pixel variance  fixed map / CCD  s0^2/F^2 + M/(G F)                (Sec. 2.1, Eq. 6)
 *                   EMCCD  E M/(G_tot F)                                (Sec. 2.1, Eq. 7)
 *   pixel loss      rho(z) + ln(sigma), z = (I - M)/sigma               (Sec. 2.3, Eq. 8;
 *                   rho = z^2/2 (Gaussian), Huber (Sec. 2.4, Eq. 12),   Sec. 2.4, Eq. 13)
 *                   Cauchy ln(1+z^2) (a Student-t drop-in, Sec. 2.4)
 *   total loss      L = sum over unmasked valid pixels
 *   gradient        dL/dK_lm = sum_p dl/dM_p R_(p+lm),  dL/db_pq = sum_p dl/dM_p eta^p xi^q
 *
 * The per-pixel curvature d2l/dM2 is exported too: because M is linear in
 * theta = [K, b], the Hessian of L is sum_p (d2l/dM2)_p phi_p phi_p^T with
 * phi_p = [R window of p, background basis at p]; the Python side forms that
 * product.  theta holds K row-major, then b_00, b_01, ..., b_0d, b_10, ...,
 * b_d0 (q fastest, the order of the double sum of Eq. 18).
 *
 * Readings of points the paper leaves open (the same ones the CUDA path takes):
 *   - with a fixed variance the ln(sigma) term is a constant and is dropped;
 *   - a model-dependent variance is clamped below at var_floor, and where it
 *     is clamped its derivative with respect to M is taken as zero;
 *   - the constant normalisation terms (N/2 ln 2pi, the Huber Q) are dropped.
 *
 * Threading: rows of the valid region are independent; each row's sums are
 * kept separately and added in row order, so the result does not depend on
 * the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* loss shapes rho(z) */
#define ORC_RHO_GAUSS 0
#define ORC_RHO_HUBER 1
#define ORC_RHO_CAUCHY 2
/* variance models */
#define ORC_VAR_FIXED 0
#define ORC_VAR_CCD 1
#define ORC_VAR_EMCCD 2

/* params[] layout (all doubles):
 *  0 rho kind, 1 variance kind, 2 sigma0 (read noise), 3 gain G (or G_total),
 *  4 excess factor E, 5 huber c, 6 scalar fixed variance (used when no map),
 *  7 variance floor                                                          */

typedef struct {
    int rho, noise;
    double sigma0, gain, excess, c, var_scalar, var_floor;
} spec_t;

static spec_t read_spec(const double *p)
{
    spec_t s;
    s.rho = (int)p[0];
    s.noise = (int)p[1];
    s.sigma0 = p[2];
    s.gain = p[3];
    s.excess = p[4];
    s.c = p[5];
    s.var_scalar = p[6];
    s.var_floor = p[7];
    return s;
}

/* Loss of one pixel and its first two derivatives with respect to M. */
static void pixel_terms(const spec_t *s, double I, double M, double vmap, double F,
                        double *ell, double *d1, double *d2, double *zout)
{
    double v, dv;
    if (s->noise == ORC_VAR_FIXED) {
        v = vmap;
        dv = 0.0;
    } else if (s->noise == ORC_VAR_CCD) {
        v = s->sigma0 * s->sigma0 / (F * F) + M / (s->gain * F);
        dv = 1.0 / (s->gain * F);
    } else {
        v = s->excess * M / (s->gain * F);
        dv = s->excess / (s->gain * F);
    }
    if (s->noise != ORC_VAR_FIXED && v < s->var_floor) {
        v = s->var_floor;
        dv = 0.0;
    }
    double sd = sqrt(v);
    double r = I - M;
    double z = r / sd;
    /* z = (I - M) v^{-1/2};  v linear in M, so d2v/dM2 = 0 */
    double dz = -1.0 / sd - 0.5 * z * dv / v;
    double d2z = dv / (v * sd) + 0.75 * z * dv * dv / (v * v);

    double rho, rho1, rho2;
    if (s->rho == ORC_RHO_GAUSS) {
        rho = 0.5 * z * z;
        rho1 = z;
        rho2 = 1.0;
    } else if (s->rho == ORC_RHO_HUBER) {
        double az = fabs(z);
        if (az <= s->c) {
            rho = 0.5 * z * z;
            rho1 = z;
            rho2 = 1.0;
        } else {
            rho = s->c * (az - 0.5 * s->c);
            rho1 = (z > 0 ? s->c : -s->c);
            rho2 = 0.0;
        }
    } else {
        double q = 1.0 + z * z;
        rho = log(q);
        rho1 = 2.0 * z / q;
        rho2 = 2.0 * (1.0 - z * z) / (q * q);
    }

    double e = rho, g1 = rho1 * dz, g2 = rho2 * dz * dz + rho1 * d2z;
    if (s->noise != ORC_VAR_FIXED) {
        /* ln(sigma) = ln(v)/2 */
        e += 0.5 * log(v);
        g1 += 0.5 * dv / v;
        g2 -= 0.5 * dv * dv / (v * v);
    }
    if (ell) *ell = e;
    if (d1) *d1 = g1;
    if (d2) *d2 = g2;
    if (zout) *zout = z;
}

/* Number of background coefficients of degree d: (d+1)(d+2)/2. */
static int n_background(int deg) { return (deg + 1) * (deg + 2) / 2; }

/* Background basis functions eta^p xi^q at full-image pixel (i, j), in the
 * coefficient order (Eq. 18, Eq. 19). */
static void background_basis(int deg, int H, int W, int i, int j, double *phi)
{
    double eta = (j - 0.5 * (W - 1)) / (double)W;
    double xi = (i - 0.5 * (H - 1)) / (double)H;
    int k = 0;
    for (int p = 0; p <= deg; ++p)
        for (int q = 0; q <= deg - p; ++q)
            phi[k++] = pow(eta, p) * pow(xi, q);
}

static double model_at(const double *R, int H, int W, int ld, int m, int deg,
                       const double *theta, int i, int j)
{
    int h = m / 2;
    double acc = 0.0, phi[64];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            acc += theta[a * m + b] * R[(size_t)(i - h + a) * ld + (j - h + b)];
    background_basis(deg, H, W, i, j, phi);
    for (int k = 0; k < n_background(deg); ++k) acc += theta[m * m + k] * phi[k];
    return acc;
}

static int check_args(int H, int W, int ld, int m)
{
    if (m < 1 || (m % 2) == 0) return -1;
    if (W < 1 || H < 1) return -1;
    if (H < m || W < m || ld < W) return -1;
    return 0;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* M over the valid region, row-major (H-2h) x (W-2h). */
int oracle_model(const double *R, int H, int W, int ld, int m, int deg, const double *theta,
                 double *M_out, int nthreads)
{
    if (check_args(H, W, ld, m) || deg < 0 || deg > 9) return -1;
    int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < Hv; ++y)
        for (int x = 0; x < Wv; ++x)
            M_out[(size_t)y * Wv + x] = model_at(R, H, W, ld, m, deg, theta, y + h, x + h);
    return 0;
}

/* Per-pixel terms over the valid region from a given model image M (valid
 * layout).  Any of the outputs may be NULL.  Masked pixels get zeros. */
int oracle_pixel_terms(const double *I, const uint8_t *mask, const double *var,
                       const double *flat, int H, int W, int ld, int m,
                       const double *params, const double *M,
                       double *ell_out, double *d1_out, double *d2_out, double *z_out)
{
    if (check_args(H, W, ld, m)) return -1;
    spec_t s = read_spec(params);
    int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h;
    for (int y = 0; y < Hv; ++y)
        for (int x = 0; x < Wv; ++x) {
            size_t q = (size_t)(y + h) * ld + (x + h), o = (size_t)y * Wv + x;
            int use = mask ? (mask[q] != 0) : 1;
            double e = 0, g1 = 0, g2 = 0, z = 0;
            double vm = var ? var[q] : s.var_scalar;
            double F = flat ? flat[q] : 1.0;
            pixel_terms(&s, I[q], M[o], vm, F, &e, &g1, &g2, &z);
            if (!use) {
                e = 0;
                g1 = 0;
                g2 = 0;
            }
            if (ell_out) ell_out[o] = e;
            if (d1_out) d1_out[o] = g1;
            if (d2_out) d2_out[o] = g2;
            if (z_out) z_out[o] = z;
        }
    return 0;
}

/* Loss and gradient (m*m + (d+1)(d+2)/2 entries: K row-major, then the
 * background coefficients) at theta. */
int oracle_loss_grad(const double *R, const double *I, const uint8_t *mask,
                     const double *var, const double *flat, int H, int W, int ld, int m,
                     int deg, const double *params, const double *theta, double *loss_out,
                     double *grad_out, int nthreads)
{
    if (check_args(H, W, ld, m) || deg < 0 || deg > 9) return -1;
    spec_t s = read_spec(params);
    int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h, nbg = n_background(deg), n = m * m + nbg;
    double *row_loss = (double *)calloc((size_t)Hv, sizeof(double));
    double *row_grad = (double *)calloc((size_t)Hv * n, sizeof(double));
    if (!row_loss || !row_grad) {
        free(row_loss);
        free(row_grad);
        return -2;
    }
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 2)
    for (int y = 0; y < Hv; ++y) {
        int i = y + h;
        double *gr = row_grad + (size_t)y * n;
        double ls = 0.0;
        for (int x = 0; x < Wv; ++x) {
            int j = x + h;
            size_t q = (size_t)i * ld + j;
            if (mask && mask[q] == 0) continue;
            double M = model_at(R, H, W, ld, m, deg, theta, i, j), phi[64];
            double e, g1;
            double vm = var ? var[q] : s.var_scalar;
            double F = flat ? flat[q] : 1.0;
            pixel_terms(&s, I[q], M, vm, F, &e, &g1, NULL, NULL);
            ls += e;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b)
                    gr[a * m + b] += g1 * R[(size_t)(i - h + a) * ld + (j - h + b)];
            background_basis(deg, H, W, i, j, phi);
            for (int k = 0; k < nbg; ++k) gr[m * m + k] += g1 * phi[k];
        }
        row_loss[y] = ls;
    }
    double L = 0.0;
    for (int k = 0; k < n; ++k) grad_out[k] = 0.0;
    for (int y = 0; y < Hv; ++y) {
        L += row_loss[y];
        for (int k = 0; k < n; ++k) grad_out[k] += row_grad[(size_t)y * n + k];
    }
    *loss_out = L;
    free(row_loss);
    free(row_grad);
    return 0;
}

/* Number of valid, unmasked pixels (N_data, Sec. 2.1). */
long long oracle_ndata(const uint8_t *mask, int H, int W, int ld, int m)
{
    if (check_args(H, W, ld, m)) return -1;
    int h = m / 2;
    long long n = 0;
    for (int i = h; i < H - h; ++i)
        for (int j = h; j < W - h; ++j)
            n += mask ? (mask[(size_t)i * ld + j] != 0) : 1;
    return n;
}

/* Design rows of the linear model for the valid-region rows [y0, y1): for
 * each valid pixel p, phi_p = [R window of p (m*m, row-major), background
 * basis at p] (Eq. 2, Eq. 18), written row after row into phi (n columns,
 * n = m*m + (d+1)(d+2)/2); if w is given (valid-region map of pitch ldw),
 * also w_p phi_p into phiw.  The Python side forms the normal matrix or the
 * Hessian sum_p w_p phi_p phi_p^T from these blocks with one matrix product;
 * this routine only lays the rows out (a parallel copy, no sums). */
int oracle_design_rows(const double *R, int H, int W, int ld, int m, int deg, int y0, int y1,
                       const double *w, int ldw, double *phi, double *phiw, int nthreads)
{
    if (check_args(H, W, ld, m) || deg < 0 || deg > 9) return -1;
    int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h;
    if (y0 < 0 || y1 > Hv || y0 > y1) return -1;
    int nb = n_background(deg), n = m * m + nb;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = y0; y < y1; ++y) {
        for (int x = 0; x < Wv; ++x) {
            double *row = phi + ((size_t)(y - y0) * Wv + x) * n;
            for (int a = 0; a < m; ++a) {
                const double *rr = R + (size_t)(y + a) * ld + x;
                for (int b = 0; b < m; ++b) row[a * m + b] = rr[b];
            }
            background_basis(deg, H, W, y + h, x + h, row + m * m);
            if (w && phiw) {
                double wp = w[(size_t)y * ldw + x];
                double *rw = phiw + ((size_t)(y - y0) * Wv + x) * n;
                for (int k = 0; k < n; ++k) rw[k] = wp * row[k];
            }
        }
    }
    return 0;
}
