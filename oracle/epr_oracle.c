/*
 * epr_oracle.c -- FP64 CPU oracle for fast eikonal phase retrieval (EPR),
 * arXiv 2601.22793 ("Fast Eikonal Phase Retrieval for High-Throughput
 * Beamlines", Mirone et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the package smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no source, header, table or helper with the CUDA path.
 *
 * Everything is double precision, single threaded, with plain loops in the
 * order the paper states the steps.  Arrays are row-major [ny][nx] with y the
 * row index, as in the paper's P_s(y, x).
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository, with the reason):
 *   R1  discrete gradient of the thickness: central differences in the
 *       interior, first-order one-sided at the edges (numpy.gradient with
 *       unit spacing), in thickness units per pixel.
 *   R2  phase of line s: phi_s = -k_s delta_s tau (Eq. 6 with Eq. 7), so the
 *       shift is Delta_s = -L delta_s grad(tau) and, in pixels,
 *       u_s = -(L delta_s / p^2) * G[tau]   (Eq. 2 in pixel units).
 *   R3  splat targets outside the detector grid are dropped (counted in
 *       `dropped`); the adjoint reads zero outside the grid.
 *   R4  the preconditioner is periodic, without padding, with the continuous
 *       symbol H_s(q) = mu_s / (mu_s + L delta_s |q|^2), |q|^2 =
 *       4 pi^2 (fx^2 + fy^2), fx = numpy.fft.fftfreq(nx, p).
 *   R5  residual split: r_s = r * P_s / P where P > 1e-30, else r * f_s.
 *   R6  projection to one thickness: least squares in the log domain with
 *       weights f_s: tau' = -sum f_s mu_s ln(I'_s/f_s) / sum f_s mu_s^2.
 *   R7  update: I'_s = max(I_s + omega * h_s, eps_I * f_s).
 *   R8  stop when kappa = |tau' - tau| / |tau'| <= tol, or after n_iter.
 *   R9  mu_s = 2 k_s beta_s, k_s = 2 pi / lambda_s, lambda_s = hc / E_s.
 *   R10 local stencils: D_i central (one-sided at edges), D_ii the compact
 *       [1, -2, 1] with replicated edges, D_ij = D_i D_j for i != j.
 *   R11 oversampled internal grid ("Results": solves on grids whose pixel is
 *       the detector pixel divided by o): the thickness and the forward model
 *       live on the fine grid (o ny) x (o nx) with pixel p / o; the model's
 *       detector image is the mean of each o x o block of the fine P; the
 *       residual D - mean(P) is formed at detector resolution and replicated
 *       to the o x o fine pixels of its block before the split, the
 *       back-transport, the preconditioner (fine grid) and the update.
 *       o = 1 is the plain solve.
 *   R12 non-local model to second order (the caption of the non-local grid
 *       figure calls the non-local model second order, while the Methods
 *       define the transport M_s as pure WKB0): P_s = M_s[I_s] minus the
 *       diffraction-pressure (WKB1) term of Eq. 1, eps^2/(4 p^4)
 *       D_i(I_s D_i Q_s), evaluated on the detector grid with the object
 *       intensity as in the local closure of order 2; the back-transport
 *       stays the transport's adjoint.  At zero shift it is the local
 *       closure of order 2.
 *   R13 x-dependent effective spectrum ("Remark on spatially varying
 *       spectra", whose file format and blockwise interpolation are in a
 *       supplement that is not available): x is the detector column; a table
 *       of knot columns gives each line's weight, delta and beta, linearly
 *       interpolated in x and constant beyond the end knots; f_s(x) is the
 *       weight normalised per column, mu_s(x) = 2 k_s beta_s(x), the shift
 *       u_s = -(L delta_s(x) / p^2) G[tau] holds the table constant under the
 *       derivative (slow variation), the update floors at eps_I f_s(x) and the
 *       projection weighs by f_s(x) mu_s(x) per column; the preconditioner,
 *       which must be FFT-diagonal, takes each line's column means of mu_s and
 *       L delta_s.
 *
 * Beyond the paper: orc_vjp (the transpose of the non-local forward model)
 * and orc_solve_vjp (reverse mode through a fixed number of iterations of
 * the non-local solve, for calibrating L, delta_s and beta_s) are pinned by
 * finite differences of the oracle's own forward and solve.
 *
 * The residual split of R5 is pinned through the paper's word for it,
 * "positivity-weighted": without transport and preconditioning (L = 0) and
 * with omega = 1 the update of line s is I_s + w_s (D - P), and the only
 * weights that sum to one and keep every line positive for every D >= 0 are
 * w_s = P_s / P (each line is then scaled by D / P).  The floor of R7 is
 * pinned by data with a dark block, where the first update from the flat
 * field falls to eps_I f_s in closed form.  Every step is pinned by the CPU
 * tests.
 */
#include <complex.h>
#undef I /* the object intensity is called I below; the imaginary unit is _Complex_I */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_HC_EV_M 1.2398419843320026e-6 /* h c in eV m */
#define ORC_PI 3.14159265358979323846

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 3 };
enum { ORC_MODEL_NONLOCAL = 0, ORC_MODEL_LOCAL1 = 1, ORC_MODEL_LOCAL2 = 2,
       ORC_MODEL_NONLOCAL_WKB1 = 3 };

#define IDX(y, x) ((size_t)(y) * (size_t)nx + (size_t)(x))

/* ------------------------------------------------------------------------ */
/* Per-line physical constants.                                             */
/* ------------------------------------------------------------------------ */

/* lambda_s = hc/E_s, k_s = 2 pi/lambda_s ("Local forward model summary":
 * k = 2 pi / lambda), mu_s = 2 k_s beta_s (attenuation of the intensity
 * |U|^2 for n = 1 - delta + i beta), f_s = weights normalised to sum 1
 * (Eq. 7, I_s already carries its spectral weight), shift coefficient
 * c_s = -L delta_s / p^2 (reading R2), eps_s = L / k_s (Eq. 2). */
int orc_line_params(int n_lines, const double* E_keV, const double* delta,
                    const double* beta, const double* weights, double L,
                    double p, double* f, double* mu, double* k, double* cshift,
                    double* eps)
{
    if (n_lines <= 0 || L < 0.0 || !(p > 0.0)) return ORC_EINVAL;
    double wsum = 0.0;
    for (int s = 0; s < n_lines; ++s) {
        if (!(E_keV[s] > 0.0) || weights[s] < 0.0) return ORC_EINVAL;
        wsum += weights[s];
    }
    if (!(wsum > 0.0)) return ORC_EINVAL;
    for (int s = 0; s < n_lines; ++s) {
        double lam = ORC_HC_EV_M / (E_keV[s] * 1e3);
        k[s] = 2.0 * ORC_PI / lam;
        mu[s] = 2.0 * k[s] * beta[s];
        f[s] = weights[s] / wsum;
        cshift[s] = -L * delta[s] / (p * p);
        eps[s] = L / k[s];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Discrete derivatives (readings R1, R10).                                 */
/* ------------------------------------------------------------------------ */

/* d/dx with unit spacing: central inside, one-sided at x = 0 and x = nx-1. */
static void d_x(int ny, int nx, const double* a, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double v;
            if (x == 0) v = a[IDX(y, 1)] - a[IDX(y, 0)];
            else if (x == nx - 1) v = a[IDX(y, nx - 1)] - a[IDX(y, nx - 2)];
            else v = 0.5 * (a[IDX(y, x + 1)] - a[IDX(y, x - 1)]);
            out[IDX(y, x)] = v;
        }
}

/* d/dy with unit spacing: central inside, one-sided at y = 0 and y = ny-1. */
static void d_y(int ny, int nx, const double* a, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double v;
            if (y == 0) v = a[IDX(1, x)] - a[IDX(0, x)];
            else if (y == ny - 1) v = a[IDX(ny - 1, x)] - a[IDX(ny - 2, x)];
            else v = 0.5 * (a[IDX(y + 1, x)] - a[IDX(y - 1, x)]);
            out[IDX(y, x)] = v;
        }
}

/* d2/dx2: [1, -2, 1] with the edge value replicated outside the grid. */
static void d_xx(int ny, int nx, const double* a, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double l = a[IDX(y, x > 0 ? x - 1 : 0)];
            double r = a[IDX(y, x < nx - 1 ? x + 1 : nx - 1)];
            out[IDX(y, x)] = l - 2.0 * a[IDX(y, x)] + r;
        }
}

/* d2/dy2: [1, -2, 1] with the edge value replicated outside the grid. */
static void d_yy(int ny, int nx, const double* a, double* out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double b = a[IDX(y > 0 ? y - 1 : 0, x)];
            double t = a[IDX(y < ny - 1 ? y + 1 : ny - 1, x)];
            out[IDX(y, x)] = b - 2.0 * a[IDX(y, x)] + t;
        }
}

/* G[tau] = (d tau/dy, d tau/dx) per pixel (reading R1). */
void orc_gradient(int ny, int nx, const double* T, double* gy, double* gx)
{
    d_y(ny, nx, T, gy);
    d_x(ny, nx, T, gx);
}

/* ------------------------------------------------------------------------ */
/* Non-local transport: bilinear redistribution and its adjoint.            */
/* ------------------------------------------------------------------------ */

/* Forward WKB0 transport of one line (Eq. 3), discretised as the paper's
 * conservative bilinear redistribution ("Discrete implementation" in the
 * non-local Methods subsection): source pixel (y, x) with mass I(y, x) goes
 * to (x_t, y_t) = (x + u_x, y + u_y); with x0 = floor(x_t), y0 = floor(y_t),
 * d_x = x_t - x0, d_y = y_t - y0 the weights are
 *   w00 = (1-d_x)(1-d_y) -> (y0,   x0)     w10 = d_x(1-d_y) -> (y0,   x0+1)
 *   w01 = (1-d_x) d_y    -> (y0+1, x0)     w11 = d_x d_y    -> (y0+1, x0+1).
 * P is ACCUMULATED (+=).  Mass whose corner lies outside the grid is added to
 * *dropped (reading R3), so sum(P) + dropped = sum(I). */
void orc_splat(int ny, int nx, const double* I, const double* uy,
               const double* ux, double* P, double* dropped)
{
    double lost = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double m = I[IDX(y, x)];
            double xt = (double)x + ux[IDX(y, x)];
            double yt = (double)y + uy[IDX(y, x)];
            double fx0 = floor(xt), fy0 = floor(yt);
            double dx = xt - fx0, dy = yt - fy0;
            double w[4] = {(1.0 - dx) * (1.0 - dy), dx * (1.0 - dy),
                           (1.0 - dx) * dy, dx * dy};
            int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
            for (int c = 0; c < 4; ++c) {
                double cx = fx0 + ox[c], cy = fy0 + oy[c];
                if (cx >= 0.0 && cx < (double)nx && cy >= 0.0 && cy < (double)ny)
                    P[IDX((int)cy, (int)cx)] += m * w[c];
                else
                    lost += m * w[c];
            }
        }
    if (dropped) *dropped += lost;
}

/* Exact adjoint of orc_splat (Eq. 4): for every object pixel, the bilinear
 * combination of the detector values e at the same four corners with the
 * same four weights; corners outside the grid contribute 0 (reading R3). */
void orc_gather(int ny, int nx, const double* e, const double* uy,
                const double* ux, double* g)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double xt = (double)x + ux[IDX(y, x)];
            double yt = (double)y + uy[IDX(y, x)];
            double fx0 = floor(xt), fy0 = floor(yt);
            double dx = xt - fx0, dy = yt - fy0;
            double w[4] = {(1.0 - dx) * (1.0 - dy), dx * (1.0 - dy),
                           (1.0 - dx) * dy, dx * dy};
            int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
            double acc = 0.0;
            for (int c = 0; c < 4; ++c) {
                double cx = fx0 + ox[c], cy = fy0 + oy[c];
                if (cx >= 0.0 && cx < (double)nx && cy >= 0.0 && cy < (double)ny)
                    acc += w[c] * e[IDX((int)cy, (int)cx)];
            }
            g[IDX(y, x)] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms.                                             */
/* ------------------------------------------------------------------------ */

/* Textbook O(n^2) DFT: X[k] = sum_j x[j] exp(sign 2 pi i j k / n). */
void orc_dft_naive(int n, const double* re, const double* im, double* ore,
                   double* oim, int sign)
{
    for (int k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            double a = sign * 2.0 * ORC_PI * (double)(((long long)j * k) % n) / n;
            double c = cos(a), s = sin(a);
            sr += re[j] * c - im[j] * s;
            si += re[j] * s + im[j] * c;
        }
        ore[k] = sr;
        oim[k] = si;
    }
}

/* Recursive decimation-in-time FFT for any n: split off the smallest prime
 * factor r of n (r = n when n is prime, which makes that level a plain DFT),
 * transform the r decimated subsequences x[q + r j] of length m = n / r, and
 * combine  X[k] = sum_q W^(q k) Y_q[k mod m],  W = exp(sign 2 pi i / n).
 * `w` holds exp(sign 2 pi i t / N) for the top-level length N, and
 * `wstride` = N / n maps this level's twiddles into it. */
static void fft_rec(int n, const double complex* in, int stride,
                    double complex* out, double complex* tmp,
                    const double complex* w, int wstride)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int r = n;
    for (int d = 2; d * d <= n; ++d)
        if (n % d == 0) {
            r = d;
            break;
        }
    int m = n / r;
    for (int q = 0; q < r; ++q)
        fft_rec(m, in + (size_t)q * stride, stride * r, tmp + (size_t)q * m,
                out + (size_t)q * m, w, wstride * r);
    for (int k = 0; k < n; ++k) {
        double complex acc = 0.0;
        for (int q = 0; q < r; ++q) {
            long long t = ((long long)q * k) % n;
            acc += w[t * wstride] * tmp[(size_t)q * m + (k % m)];
        }
        out[k] = acc;
    }
    /* tmp is scratch for this level only; the caller's copy is in out. */
}

/* In-place unnormalised 1-D FFT, sign -1 forward (numpy.fft.fft), +1 inverse
 * without the 1/n factor. */
int orc_fft(int n, double* re, double* im, int sign)
{
    if (n <= 0) return ORC_EINVAL;
    double complex* a = malloc(sizeof(double complex) * (size_t)n);
    double complex* b = malloc(sizeof(double complex) * (size_t)n);
    double complex* c = malloc(sizeof(double complex) * (size_t)n);
    double complex* w = malloc(sizeof(double complex) * (size_t)n);
    if (!a || !b || !c || !w) {
        free(a); free(b); free(c); free(w);
        return ORC_ENOMEM;
    }
    for (int t = 0; t < n; ++t) {
        double ang = sign * 2.0 * ORC_PI * (double)t / n;
        w[t] = cos(ang) + _Complex_I * sin(ang);
        a[t] = re[t] + _Complex_I * im[t];
    }
    fft_rec(n, a, 1, b, c, w, 1);
    for (int t = 0; t < n; ++t) {
        re[t] = creal(b[t]);
        im[t] = cimag(b[t]);
    }
    free(a); free(b); free(c); free(w);
    return ORC_OK;
}

/* 2-D transform: all rows, then all columns (separable DFT). */
int orc_fft2(int ny, int nx, double* re, double* im, int sign)
{
    int nmax = nx > ny ? nx : ny;
    double* lr = malloc(sizeof(double) * (size_t)nmax);
    double* li = malloc(sizeof(double) * (size_t)nmax);
    if (!lr || !li) {
        free(lr); free(li);
        return ORC_ENOMEM;
    }
    int st = ORC_OK;
    for (int y = 0; y < ny && st == ORC_OK; ++y) {
        for (int x = 0; x < nx; ++x) {
            lr[x] = re[IDX(y, x)];
            li[x] = im[IDX(y, x)];
        }
        st = orc_fft(nx, lr, li, sign);
        for (int x = 0; x < nx; ++x) {
            re[IDX(y, x)] = lr[x];
            im[IDX(y, x)] = li[x];
        }
    }
    for (int x = 0; x < nx && st == ORC_OK; ++x) {
        for (int y = 0; y < ny; ++y) {
            lr[y] = re[IDX(y, x)];
            li[y] = im[IDX(y, x)];
        }
        st = orc_fft(ny, lr, li, sign);
        for (int y = 0; y < ny; ++y) {
            re[IDX(y, x)] = lr[y];
            im[IDX(y, x)] = li[y];
        }
    }
    free(lr); free(li);
    return st;
}

/* numpy.fft.fftfreq(n, d)[k]: k / (n d) for k < (n + 1) / 2, else (k - n) / (n d). */
static double fftfreq(int n, double d, int k)
{
    int kk = (k < (n + 1) / 2) ? k : k - n;
    return (double)kk / ((double)n * d);
}

/* FFT-diagonal Paganin-type preconditioner P_{1,s}^{-1} ("Linear term and
 * relation to Paganin"; "Iteration structure"): g <- Re F^-1[ H F[g] ] with
 * H(q) = mu / (mu + L delta |q|^2) (reading R4), in place. */
int orc_paganin(int ny, int nx, double p, double mu, double Ldelta, double* g)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* im = calloc(n, sizeof(double));
    if (!im) return ORC_ENOMEM;
    int st = orc_fft2(ny, nx, g, im, -1);
    if (st == ORC_OK) {
        for (int y = 0; y < ny; ++y) {
            double fy = fftfreq(ny, p, y);
            for (int x = 0; x < nx; ++x) {
                double fx = fftfreq(nx, p, x);
                double q2 = 4.0 * ORC_PI * ORC_PI * (fx * fx + fy * fy);
                double H = mu / (mu + Ldelta * q2);
                g[IDX(y, x)] *= H;
                im[IDX(y, x)] *= H;
            }
        }
        st = orc_fft2(ny, nx, g, im, +1);
        for (size_t i = 0; i < n; ++i) g[i] /= (double)n;
    }
    free(im);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Forward models.                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_lines;
    double p, L;
    double *f, *mu, *k, *c, *eps, *delta;
} orc_lines;

static int lines_init(orc_lines* ln, int n_lines, const double* E_keV,
                      const double* delta, const double* beta,
                      const double* weights, double L, double p)
{
    memset(ln, 0, sizeof(*ln));
    ln->n_lines = n_lines;
    ln->p = p;
    ln->L = L;
    size_t b = sizeof(double) * (size_t)(n_lines > 0 ? n_lines : 1);
    ln->f = malloc(b); ln->mu = malloc(b); ln->k = malloc(b);
    ln->c = malloc(b); ln->eps = malloc(b); ln->delta = malloc(b);
    if (!ln->f || !ln->mu || !ln->k || !ln->c || !ln->eps || !ln->delta)
        return ORC_ENOMEM;
    for (int s = 0; s < n_lines; ++s) ln->delta[s] = delta[s];
    return orc_line_params(n_lines, E_keV, delta, beta, weights, L, p, ln->f,
                           ln->mu, ln->k, ln->c, ln->eps);
}

static void lines_free(orc_lines* ln)
{
    free(ln->f); free(ln->mu); free(ln->k);
    free(ln->c); free(ln->eps); free(ln->delta);
}

/* The diffraction-pressure (WKB1) term of Eq. 1 in pixel units, subtracted
 * from P: P -= eps^2/(4 p^4) [D_x(I D_x Q) + D_y(I D_y Q)] with
 * Q = (D_xx + D_yy) sqrt(I) / sqrt(I) (reading R10 for the stencils). */
static int wkb1_term(int ny, int nx, const double* I, double eps, double p, double* P)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* a = malloc(sizeof(double) * n);
    double* b = malloc(sizeof(double) * n);
    double* t = malloc(sizeof(double) * n);
    double* q = malloc(sizeof(double) * n);
    if (!a || !b || !t || !q) {
        free(a); free(b); free(t); free(q);
        return ORC_ENOMEM;
    }
    for (size_t i = 0; i < n; ++i) a[i] = sqrt(I[i]);
    d_xx(ny, nx, a, b);
    d_yy(ny, nx, a, t);
    for (size_t i = 0; i < n; ++i) q[i] = (a[i] > 0.0) ? (b[i] + t[i]) / a[i] : 0.0;
    double coef = eps * eps / (4.0 * p * p * p * p);
    d_x(ny, nx, q, a);
    for (size_t i = 0; i < n; ++i) a[i] *= I[i];
    d_x(ny, nx, a, b);
    for (size_t i = 0; i < n; ++i) P[i] -= coef * b[i];
    d_y(ny, nx, q, a);
    for (size_t i = 0; i < n; ++i) a[i] *= I[i];
    d_y(ny, nx, a, b);
    for (size_t i = 0; i < n; ++i) P[i] -= coef * b[i];
    free(a); free(b); free(t); free(q);
    return ORC_OK;
}

/* Local O(L^2) closure of one line (Eq. 1 in pixel units, reading R10):
 *   P = I - D_i(I u_i)                                             (m = 1)
 *       + 1/2 D_i D_j (I u_i u_j) - eps^2/(4 p^4) D_i(I D_i Q)    (m = 2)
 * with Q = (D_xx + D_yy) sqrt(I) / sqrt(I) (Q of Eq. 1 in pixel units).
 * The physical derivative is D/p and eps grad(phi) = p u, which turns the
 * eps and eps^2/2 terms of Eq. 1 into the pixel forms above and leaves
 * eps^2 / (4 p^4) in front of the diffraction-pressure term. */
static int local_line(int ny, int nx, int order, const double* I,
                      const double* uy, const double* ux, double eps, double p,
                      double* P)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* a = malloc(sizeof(double) * n);
    double* b = malloc(sizeof(double) * n);
    double* t = malloc(sizeof(double) * n);
    double* q = malloc(sizeof(double) * n);
    if (!a || !b || !t || !q) {
        free(a); free(b); free(t); free(q);
        return ORC_ENOMEM;
    }
    for (size_t i = 0; i < n; ++i) P[i] = I[i];
    /* - D_x(I u_x) - D_y(I u_y) */
    for (size_t i = 0; i < n; ++i) a[i] = I[i] * ux[i];
    d_x(ny, nx, a, b);
    for (size_t i = 0; i < n; ++i) P[i] -= b[i];
    for (size_t i = 0; i < n; ++i) a[i] = I[i] * uy[i];
    d_y(ny, nx, a, b);
    for (size_t i = 0; i < n; ++i) P[i] -= b[i];
    if (order >= 2) {
        /* + 1/2 [ D_xx(I ux^2) + 2 D_x D_y(I ux uy) + D_yy(I uy^2) ] */
        for (size_t i = 0; i < n; ++i) a[i] = I[i] * ux[i] * ux[i];
        d_xx(ny, nx, a, b);
        for (size_t i = 0; i < n; ++i) P[i] += 0.5 * b[i];
        for (size_t i = 0; i < n; ++i) a[i] = I[i] * uy[i] * uy[i];
        d_yy(ny, nx, a, b);
        for (size_t i = 0; i < n; ++i) P[i] += 0.5 * b[i];
        for (size_t i = 0; i < n; ++i) a[i] = I[i] * ux[i] * uy[i];
        d_y(ny, nx, a, t);
        d_x(ny, nx, t, b);
        for (size_t i = 0; i < n; ++i) P[i] += b[i];
        /* - eps^2/(4 p^4) [ D_x(I D_x Q) + D_y(I D_y Q) ] */
        free(a); free(b); free(t); free(q);
        return wkb1_term(ny, nx, I, eps, p, P);
    }
    free(a); free(b); free(t); free(q);
    return ORC_OK;
}

/* Polychromatic forward (Eq. 5): P = sum_s F_s[I_s] with I_s = f_s exp(-mu_s
 * tau) (Eq. 7) and u_s = c_s G[tau] (reading R2).  F_s is the bilinear
 * redistribution for model 0 and the local closure of order m for models 1, 2.
 * Model 3 (reading R12) is the non-local model to second order: the bilinear
 * redistribution (WKB0 transport, all orders of the shift) minus the
 * diffraction-pressure term of Eq. 1, evaluated on the detector grid with the
 * line's object intensity, as the local closure of order 2 evaluates it.
 * Ps (n_lines maps, may be NULL) and dropped (n_lines values, may be NULL)
 * receive the per-line predictions and the per-line mass that left the grid. */
static int forward_impl(int ny, int nx, const orc_lines* ln, int model,
                        const double* T, double* P, double* Ps, double* dropped,
                        double* gy, double* gx, double* uy, double* ux,
                        double* I, double* Pl)
{
    size_t n = (size_t)nx * (size_t)ny;
    orc_gradient(ny, nx, T, gy, gx);
    for (size_t i = 0; i < n; ++i) P[i] = 0.0;
    for (int s = 0; s < ln->n_lines; ++s) {
        for (size_t i = 0; i < n; ++i) {
            uy[i] = ln->c[s] * gy[i];
            ux[i] = ln->c[s] * gx[i];
            I[i] = ln->f[s] * exp(-ln->mu[s] * T[i]);
            Pl[i] = 0.0;
        }
        double lost = 0.0;
        if (model == ORC_MODEL_NONLOCAL || model == ORC_MODEL_NONLOCAL_WKB1) {
            orc_splat(ny, nx, I, uy, ux, Pl, &lost);
            if (model == ORC_MODEL_NONLOCAL_WKB1) {
                int st = wkb1_term(ny, nx, I, ln->eps[s], ln->p, Pl);
                if (st != ORC_OK) return st;
            }
        } else {
            int st = local_line(ny, nx, model, I, uy, ux, ln->eps[s], ln->p, Pl);
            if (st != ORC_OK) return st;
        }
        for (size_t i = 0; i < n; ++i) P[i] += Pl[i];
        if (Ps) memcpy(Ps + (size_t)s * n, Pl, sizeof(double) * n);
        if (dropped) dropped[s] = lost;
    }
    return ORC_OK;
}

static double* alloc_n(size_t n) { return malloc(sizeof(double) * (n ? n : 1)); }

int orc_forward(int ny, int nx, double p, double L, int n_lines,
                const double* E_keV, const double* delta, const double* beta,
                const double* weights, int model, const double* T, double* P,
                double* Ps, double* dropped)
{
    if (ny < 2 || nx < 2 || model < 0 || model > 3) return ORC_EINVAL;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *I = alloc_n(n), *Pl = alloc_n(n);
    if (st == ORC_OK && (!gy || !gx || !uy || !ux || !I || !Pl)) st = ORC_ENOMEM;
    if (st == ORC_OK)
        st = forward_impl(ny, nx, &ln, model, T, P, Ps, dropped, gy, gx, uy, ux, I, Pl);
    free(gy); free(gx); free(uy); free(ux); free(I); free(Pl);
    lines_free(&ln);
    return st;
}

/* Non-local forward of an object whose phase and attenuation are not one
 * thickness (several materials, the data side of a single-material
 * retrieval): per line s the phase line integral Phi_s = sum_m delta_{m,s} t_m
 * and the attenuation line integral A_s = sum_m mu_{m,s} t_m (maps
 * [n_lines][ny][nx], t_m the chord through material m).  The object intensity
 * is I_s = f_s exp(-A_s) and the phase phi_s = -k_s Phi_s (Eq. 6 before the
 * single-material substitution of Eq. 7), so the shift in pixels is
 * u_s = -(L / p^2) G[Phi_s] (Eq. 2, reading R2 without tau), and
 * P = sum_s M_s[I_s] (Eqs. 3 and 5).  f_s = weights normalised to sum 1.
 * With one material (Phi_s = delta_s tau, A_s = mu_s tau) this is the
 * non-local orc_forward. */
int orc_forward_fields(int ny, int nx, double p, double L, int n_lines, const double* weights,
                       const double* Phi, const double* A, double* P, double* Ps,
                       double* dropped)
{
    if (ny < 2 || nx < 2 || n_lines < 1 || L < 0.0 || !(p > 0.0)) return ORC_EINVAL;
    double wsum = 0.0;
    for (int s = 0; s < n_lines; ++s) {
        if (weights[s] < 0.0) return ORC_EINVAL;
        wsum += weights[s];
    }
    if (!(wsum > 0.0)) return ORC_EINVAL;
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *I = alloc_n(n), *Pl = alloc_n(n);
    int st = (!gy || !gx || !uy || !ux || !I || !Pl) ? ORC_ENOMEM : ORC_OK;
    if (st == ORC_OK) {
        const double c = -L / (p * p);
        for (size_t i = 0; i < n; ++i) P[i] = 0.0;
        for (int s = 0; s < n_lines; ++s) {
            const double* ph = Phi + (size_t)s * n;
            const double* at = A + (size_t)s * n;
            const double fs = weights[s] / wsum;
            orc_gradient(ny, nx, ph, gy, gx);
            for (size_t i = 0; i < n; ++i) {
                uy[i] = c * gy[i];
                ux[i] = c * gx[i];
                I[i] = fs * exp(-at[i]);
                Pl[i] = 0.0;
            }
            double lost = 0.0;
            orc_splat(ny, nx, I, uy, ux, Pl, &lost);
            for (size_t i = 0; i < n; ++i) P[i] += Pl[i];
            if (Ps) memcpy(Ps + (size_t)s * n, Pl, sizeof(double) * n);
            if (dropped) dropped[s] = lost;
        }
    }
    free(gy); free(gx); free(uy); free(ux); free(I); free(Pl);
    return st;
}

/* Adjoint of the non-local forward for one line and fixed tau: the gather of
 * the detector map e at the line's mapped coordinates (Eq. 4). */
int orc_adjoint(int ny, int nx, double p, double L, int n_lines,
                const double* E_keV, const double* delta, const double* beta,
                const double* weights, int line, const double* T,
                const double* e, double* g)
{
    if (ny < 2 || nx < 2 || line < 0 || line >= n_lines) return ORC_EINVAL;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n);
    if (st == ORC_OK && (!gy || !gx || !uy || !ux)) st = ORC_ENOMEM;
    if (st == ORC_OK) {
        orc_gradient(ny, nx, T, gy, gx);
        for (size_t i = 0; i < n; ++i) {
            uy[i] = ln.c[line] * gy[i];
            ux[i] = ln.c[line] * gx[i];
        }
        orc_gather(ny, nx, e, uy, ux, g);
    }
    free(gy); free(gx); free(uy); free(ux);
    lines_free(&ln);
    return st;
}

/* Preconditioner of one line on a real map, in place (reading R4). */
int orc_precondition(int ny, int nx, double p, double L, int n_lines,
                     const double* E_keV, const double* delta,
                     const double* beta, const double* weights, int line,
                     double* g)
{
    if (ny < 1 || nx < 1 || line < 0 || line >= n_lines) return ORC_EINVAL;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    if (st == ORC_OK) st = orc_paganin(ny, nx, p, ln.mu[line], L * ln.delta[line], g);
    lines_free(&ln);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian product of the non-local forward (not in the paper; the  */
/* analytic transpose of Eq. 3 with Eq. 2, 6, 7 as read in R1, R2, R9).      */
/* ------------------------------------------------------------------------ */

/* Transpose of the unit-spacing numpy-gradient stencil along one axis of
 * length n (>= 3), applied to v with stride `st` over n entries starting at
 * v0: out[x] = sum_j dG[j]/da[x] v[j]. */
static double gT(const double* v0, size_t st, int n, int x)
{
    double acc = 0.0;
    /* interior rows j = x-1 (coefficient +1/2) and j = x+1 (-1/2) */
    if (x - 1 >= 1 && x - 1 <= n - 2) acc += 0.5 * v0[(size_t)(x - 1) * st];
    if (x + 1 >= 1 && x + 1 <= n - 2) acc -= 0.5 * v0[(size_t)(x + 1) * st];
    /* one-sided edges: G[0] = a[1] - a[0], G[n-1] = a[n-1] - a[n-2] */
    if (x == 1) acc += v0[0];
    if (x == 0) acc -= v0[0];
    if (x == n - 1) acc += v0[(size_t)(n - 1) * st];
    if (x == n - 2) acc -= v0[(size_t)(n - 1) * st];
    return acc;
}

/* Given gbar = dF/dP, returns Tbar = dF/dtau, and per line dF/ddelta_s,
 * dF/dbeta_s and dF/dL.  Per line s and source pixel with mapped point
 * (x + u_x, y + u_y) and corner values g00, g10, g01, g11 of gbar (0 outside
 * the grid):
 *   through I_s = f_s exp(-mu_s tau):  -mu_s I_s (M_s^* gbar)
 *   through u_s = c_s G[tau]:          c_s G^T[ubar_s], with the derivative of
 *     the bilinear weights in the target coordinates,
 *     ubar_x = I_s [(1-d_y)(g10 - g00) + d_y (g11 - g01)],
 *     ubar_y = I_s [(1-d_x)(g01 - g00) + d_x (g11 - g10)]
 *   (the right derivative where a target crosses an integer);
 *   scalars: c_s = -L delta_s / p^2 gives cbar_s = <ubar_s, G[tau]>,
 *   deltabar_s = -L / p^2 cbar_s, Lbar = sum_s -delta_s / p^2 cbar_s;
 *   mu_s = 2 k_s beta_s gives mubar_s = -<tau I_s, M_s^* gbar>, betabar_s =
 *   2 k_s mubar_s. */
int orc_vjp(int ny, int nx, double p, double L, int n_lines, const double* E_keV,
            const double* delta, const double* beta, const double* weights,
            const double* T, const double* gbar, double* Tbar, double* delta_bar,
            double* beta_bar, double* L_bar)
{
    if (ny < 3 || nx < 3) return ORC_EINVAL;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *vy = alloc_n(n), *vx = alloc_n(n);
    if (st == ORC_OK && (!gy || !gx || !vy || !vx)) st = ORC_ENOMEM;
    if (st == ORC_OK) {
        orc_gradient(ny, nx, T, gy, gx);
        for (size_t i = 0; i < n; ++i) {
            Tbar[i] = 0.0;
            vy[i] = 0.0;
            vx[i] = 0.0;
        }
        double lbar = 0.0;
        for (int s = 0; s < ln.n_lines; ++s) {
            double cbar = 0.0, mubar = 0.0;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(y, x);
                    double ux = ln.c[s] * gx[i], uy = ln.c[s] * gy[i];
                    double xt = (double)x + ux, yt = (double)y + uy;
                    double fx0 = floor(xt), fy0 = floor(yt);
                    double dx = xt - fx0, dy = yt - fy0;
                    double g[4];
                    int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
                    for (int c = 0; c < 4; ++c) {
                        double cx = fx0 + ox[c], cy = fy0 + oy[c];
                        g[c] = (cx >= 0.0 && cx < (double)nx && cy >= 0.0 && cy < (double)ny)
                                   ? gbar[IDX((int)cy, (int)cx)]
                                   : 0.0;
                    }
                    double a = (1.0 - dx) * (1.0 - dy) * g[0] + dx * (1.0 - dy) * g[1] +
                               (1.0 - dx) * dy * g[2] + dx * dy * g[3];
                    double Is = ln.f[s] * exp(-ln.mu[s] * T[i]);
                    Tbar[i] += -ln.mu[s] * Is * a;
                    double ubx = Is * ((1.0 - dy) * (g[1] - g[0]) + dy * (g[3] - g[2]));
                    double uby = Is * ((1.0 - dx) * (g[2] - g[0]) + dx * (g[3] - g[1]));
                    vx[i] += ln.c[s] * ubx;
                    vy[i] += ln.c[s] * uby;
                    cbar += ubx * gx[i] + uby * gy[i];
                    mubar += -T[i] * Is * a;
                }
            if (delta_bar) delta_bar[s] = -L / (p * p) * cbar;
            if (beta_bar) beta_bar[s] = 2.0 * ln.k[s] * mubar;
            lbar += -ln.delta[s] / (p * p) * cbar;
        }
        if (L_bar) *L_bar = lbar;
        /* G^T of the accumulated shift adjoints */
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                Tbar[IDX(y, x)] += gT(vx + IDX(y, 0), 1, nx, x);
                Tbar[IDX(y, x)] += gT(vy + x, (size_t)nx, ny, y);
            }
    }
    free(gy); free(gx); free(vy); free(vx);
    lines_free(&ln);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Iterative inversion ("Iterative inversion (local and non-local)").       */
/* ------------------------------------------------------------------------ */

/* One projection.  Per iteration n, in the order of "Iteration structure":
 *   1. per-line predictions P_s and their sum P (forward_impl);
 *   2. detector residual r = D - P, rho_n = |r| / |D|;
 *   3. split across lines, r_s = r P_s / P (reading R5);
 *   4. back-transport: g_s = M_s^* r_s (Eq. 4) for the non-local model, the
 *      identity for the local closure;
 *   5. preconditioner h_s = P_{1,s}^{-1} g_s (reading R4);
 *   6. update I'_s = max(I_s + omega h_s, eps_I f_s) (reading R7) and
 *      projection to the single-thickness form of Eq. 7 (reading R6);
 *   7. kappa_n = |tau' - tau| / |tau'|; stop when kappa_n <= tol (R8).
 * T holds the initial thickness on entry (zeros = start from flat field) and
 * the result on return.  rho and kappa (n_iter values each, may be NULL)
 * receive the history; *iters the number of iterations run. */
/* The solver of "Iteration structure" on a grid oversampled by os (R11):
 * ny, nx and p are the FINE grid's; D is [ny/os][nx/os] at detector
 * resolution; os = 1 is the plain solve. */
static int solve_impl(int ny, int nx, int os, double p, double L, int n_lines,
                      const double* E_keV, const double* delta, const double* beta,
                      const double* weights, int model, const double* D, double* T,
                      int n_iter, double omega, double tol, double eps_I, double* rho,
                      double* kappa, int* iters)
{
    if (ny < 2 || nx < 2 || model < 0 || model > 3 || n_iter < 0 || os < 1 ||
        ny % os != 0 || nx % os != 0)
        return ORC_EINVAL;
    const int nyd = ny / os, nxd = nx / os;
    const size_t nd = (size_t)nxd * (size_t)nyd;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    size_t n = (size_t)nx * (size_t)ny;
    int ns = n_lines;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *I = alloc_n(n), *Pl = alloc_n(n), *P = alloc_n(n), *r = alloc_n(n),
           *rs = alloc_n(n), *g = alloc_n(n), *num = alloc_n(n),
           *Ps = alloc_n(n * (size_t)ns);
    if (st == ORC_OK && (!gy || !gx || !uy || !ux || !I || !Pl || !P || !r ||
                         !rs || !g || !num || !Ps))
        st = ORC_ENOMEM;
    double den = 0.0;
    if (st == ORC_OK)
        for (int s = 0; s < ns; ++s) den += ln.f[s] * ln.mu[s] * ln.mu[s];
    if (st == ORC_OK && !(den > 0.0)) st = ORC_EINVAL;
    double dnorm = 0.0;
    for (size_t i = 0; st == ORC_OK && i < nd; ++i) dnorm += D[i] * D[i];
    dnorm = sqrt(dnorm);
    int it = 0;
    for (; st == ORC_OK && it < n_iter; ++it) {
        /* 1. forward */
        st = forward_impl(ny, nx, &ln, model, T, P, Ps, NULL, gy, gx, uy, ux, I, Pl);
        if (st != ORC_OK) break;
        /* 2. residual at detector resolution (the mean of each os x os block
         * of the fine model), replicated to the fine pixels of its block */
        double rr = 0.0;
        for (int yd = 0; yd < nyd; ++yd)
            for (int xd = 0; xd < nxd; ++xd) {
                double m = 0.0;
                for (int a = 0; a < os; ++a)
                    for (int b = 0; b < os; ++b) m += P[IDX(yd * os + a, xd * os + b)];
                m /= (double)os * (double)os;
                const double rd = D[(size_t)yd * nxd + xd] - m;
                rr += rd * rd;
                for (int a = 0; a < os; ++a)
                    for (int b = 0; b < os; ++b) r[IDX(yd * os + a, xd * os + b)] = rd;
            }
        if (rho) rho[it] = dnorm > 0.0 ? sqrt(rr) / dnorm : sqrt(rr);
        for (size_t i = 0; i < n; ++i) num[i] = 0.0;
        for (int s = 0; s < ns; ++s) {
            if (ln.f[s] == 0.0) continue; /* a line without weight carries nothing */
            const double* P_s = Ps + (size_t)s * n;
            /* 3. split */
            for (size_t i = 0; i < n; ++i)
                rs[i] = (P[i] > 1e-30) ? r[i] * P_s[i] / P[i] : r[i] * ln.f[s];
            /* 4. back-transport (shift of this line recomputed from tau); the
             * non-local models take the transport's adjoint (Eq. 4), the
             * local closures the identity */
            if (model == ORC_MODEL_NONLOCAL || model == ORC_MODEL_NONLOCAL_WKB1) {
                for (size_t i = 0; i < n; ++i) {
                    uy[i] = ln.c[s] * gy[i];
                    ux[i] = ln.c[s] * gx[i];
                }
                orc_gather(ny, nx, rs, uy, ux, g);
            } else {
                memcpy(g, rs, sizeof(double) * n);
            }
            /* 5. preconditioner */
            st = orc_paganin(ny, nx, p, ln.mu[s], L * ln.delta[s], g);
            if (st != ORC_OK) break;
            /* 6. update of the line and its share of the projection */
            for (size_t i = 0; i < n; ++i) {
                double Is = ln.f[s] * exp(-ln.mu[s] * T[i]);
                double In = Is + omega * g[i];
                double fl = eps_I * ln.f[s];
                if (In < fl) In = fl;
                num[i] += ln.f[s] * ln.mu[s] * log(In / ln.f[s]);
            }
        }
        if (st != ORC_OK) break;
        double dd = 0.0, tt = 0.0;
        for (size_t i = 0; i < n; ++i) {
            double tn = -num[i] / den;
            dd += (tn - T[i]) * (tn - T[i]);
            tt += tn * tn;
            T[i] = tn;
        }
        /* 7. convergence */
        double kap = tt > 0.0 ? sqrt(dd / tt) : sqrt(dd);
        if (kappa) kappa[it] = kap;
        if (kap <= tol) {
            ++it;
            break;
        }
    }
    if (iters) *iters = it;
    free(gy); free(gx); free(uy); free(ux); free(I); free(Pl); free(P);
    free(r); free(rs); free(g); free(num); free(Ps);
    lines_free(&ln);
    return st;
}

int orc_solve(int ny, int nx, double p, double L, int n_lines,
              const double* E_keV, const double* delta, const double* beta,
              const double* weights, int model, const double* D, double* T,
              int n_iter, double omega, double tol, double eps_I, double* rho,
              double* kappa, int* iters)
{
    return solve_impl(ny, nx, 1, p, L, n_lines, E_keV, delta, beta, weights, model, D, T,
                      n_iter, omega, tol, eps_I, rho, kappa, iters);
}

/* The solve on a grid oversampled by os (R11): D is the detector image
 * [nyd][nxd] with pixel p_det; T is the fine thickness [os nyd][os nxd]. */
int orc_solve_os(int nyd, int nxd, int os, double p_det, double L, int n_lines,
                 const double* E_keV, const double* delta, const double* beta,
                 const double* weights, int model, const double* D, double* T,
                 int n_iter, double omega, double tol, double eps_I, double* rho,
                 double* kappa, int* iters)
{
    if (os < 1 || !(p_det > 0.0)) return ORC_EINVAL;
    return solve_impl(nyd * os, nxd * os, os, p_det / os, L, n_lines, E_keV, delta, beta,
                      weights, model, D, T, n_iter, omega, tol, eps_I, rho, kappa, iters);
}

/* Detector image of a fine map: the mean of each os x os block (R11). */
void orc_bin(int nyd, int nxd, int os, const double* fine, double* det)
{
    const int nx = nxd * os;
    for (int yd = 0; yd < nyd; ++yd)
        for (int xd = 0; xd < nxd; ++xd) {
            double m = 0.0;
            for (int a = 0; a < os; ++a)
                for (int b = 0; b < os; ++b) m += fine[IDX(yd * os + a, xd * os + b)];
            det[(size_t)yd * nxd + xd] = m / ((double)os * (double)os);
        }
}

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian product of the unrolled non-local solve (not in the      */
/* paper: calibration of L, delta_s and beta_s by gradient descent through  */
/* a fixed number of iterations of "Iteration structure", with the readings */
/* R1-R7 of the forward solve).                                             */
/* ------------------------------------------------------------------------ */

/* out = Re F^-1[K F[in]] with the preconditioner's symbol (kind 0:
 * K = H = mu / (mu + Ld |q|^2)) or one of its partial derivatives (kind 1:
 * dH/dmu = Ld |q|^2 / (mu + Ld |q|^2)^2; kind 2: dH/dLd = -mu |q|^2 /
 * (mu + Ld |q|^2)^2), periodic and normalised as orc_paganin (reading R4).
 * K is real and even in q, so each of these operators is self-adjoint. */
static int filter_kind(int ny, int nx, double p, double mu, double Ld, int kind,
                       const double* in, double* out)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* im = calloc(n, sizeof(double));
    if (!im) return ORC_ENOMEM;
    memcpy(out, in, sizeof(double) * n);
    int st = orc_fft2(ny, nx, out, im, -1);
    if (st == ORC_OK) {
        for (int y = 0; y < ny; ++y) {
            double fy = fftfreq(ny, p, y);
            for (int x = 0; x < nx; ++x) {
                double fx = fftfreq(nx, p, x);
                double q2 = 4.0 * ORC_PI * ORC_PI * (fx * fx + fy * fy);
                double d = mu + Ld * q2;
                double K = kind == 0 ? mu / d : kind == 1 ? Ld * q2 / (d * d) : -mu * q2 / (d * d);
                out[IDX(y, x)] *= K;
                im[IDX(y, x)] *= K;
            }
        }
        st = orc_fft2(ny, nx, out, im, +1);
        for (size_t i = 0; i < n; ++i) out[i] /= (double)n;
    }
    free(im);
    return st;
}

/* Bilinear interpolation of e at the mapped point of pixel (y, x) (the
 * weights of orc_splat / orc_gather; corners outside the grid read 0) and
 * its derivatives with respect to the shift components u_x, u_y (the right
 * derivative where the point crosses an integer). */
static void interp_du(int ny, int nx, const double* e, int y, int x, double uy, double ux,
                      double* val, double* dux, double* duy)
{
    double xt = (double)x + ux, yt = (double)y + uy;
    double fx0 = floor(xt), fy0 = floor(yt);
    double dx = xt - fx0, dy = yt - fy0;
    double g[4];
    int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
    for (int c = 0; c < 4; ++c) {
        double cx = fx0 + ox[c], cy = fy0 + oy[c];
        g[c] = (cx >= 0.0 && cx < (double)nx && cy >= 0.0 && cy < (double)ny)
                   ? e[IDX((int)cy, (int)cx)]
                   : 0.0;
    }
    *val = (1.0 - dx) * (1.0 - dy) * g[0] + dx * (1.0 - dy) * g[1] + (1.0 - dx) * dy * g[2] +
           dx * dy * g[3];
    *dux = (1.0 - dy) * (g[1] - g[0]) + dy * (g[3] - g[2]);
    *duy = (1.0 - dx) * (g[2] - g[0]) + dx * (g[3] - g[1]);
}

/* Given Tbar = dF/dtau_N for tau_N, the thickness after n_iter iterations of
 * the non-local solve from T0 (zeros when NULL) with data D, relaxation omega
 * and floor eps_I (no early stop), returns dF/dT0, dF/dD, dF/ddelta_s,
 * dF/dbeta_s and dF/dL (each output may be NULL).  The iterates are stored
 * and every iteration is undone in reverse order, step by step against its
 * forward (the solver above, with the split of R5, the floor of R7 and the
 * projection of R6):
 *   tau' = -num / den, num = sum_s f_s mu_s ln(I'_s / f_s), den = sum_s f_s mu_s^2;
 *   I'_s = max(I_s + omega h_s, eps_I f_s) (no gradient through the floor);
 *   h_s = F^-1 H_s F g_s (self-adjoint; H_s depends on mu_s and L delta_s);
 *   g_s = M_s^* r_s: r_s receives the splat of the adjoint of g_s, the shift
 *     the derivative of the bilinear interpolation of r_s;
 *   r_s = r P_s / P (P > 1e-30, else r f_s), r = D - P, P = sum_s P_s;
 *   P_s = M_s[I_s]: I_s receives the gather, the shift I_s times the
 *     derivative of the interpolation of the adjoint of P_s;
 *   I_s = f_s exp(-mu_s tau), u_s = c_s G[tau], c_s = -L delta_s / p^2,
 *   mu_s = 2 k_s beta_s. */
int orc_solve_vjp(int ny, int nx, double p, double L, int n_lines, const double* E_keV,
                  const double* delta, const double* beta, const double* weights,
                  const double* D, const double* T0, int n_iter, double omega, double eps_I,
                  const double* Tbar_N, double* T0_bar, double* D_bar, double* delta_bar,
                  double* beta_bar, double* L_bar)
{
    if (ny < 3 || nx < 3 || n_iter < 0) return ORC_EINVAL;
    orc_lines ln;
    int st = lines_init(&ln, n_lines, E_keV, delta, beta, weights, L, p);
    const size_t n = (size_t)nx * (size_t)ny;
    const int ns = n_lines;
    const size_t nsn = (size_t)(ns > 0 ? ns : 1) * n;
    double* Ts = alloc_n((size_t)(n_iter + 1) * n);
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *Iw = alloc_n(n), *Pl = alloc_n(n), *P = alloc_n(n), *r = alloc_n(n),
           *num = alloc_n(n), *tb = alloc_n(n), *tn = alloc_n(n), *Pbar = alloc_n(n),
           *rbar = alloc_n(n), *vx = alloc_n(n), *vy = alloc_n(n), *hb = alloc_n(n),
           *gb = alloc_n(n), *tmp = alloc_n(n), *Db = alloc_n(n);
    double *Ps = alloc_n(nsn), *Is = alloc_n(nsn), *rs = alloc_n(nsn), *ga = alloc_n(nsn),
           *In = alloc_n(nsn), *rsb = alloc_n(nsn), *uxb = alloc_n(nsn), *uyb = alloc_n(nsn),
           *Isb = alloc_n(nsn), *Psb = alloc_n(nsn);
    double *mub = calloc((size_t)(ns > 0 ? ns : 1), sizeof(double)),
           *Ldb = calloc((size_t)(ns > 0 ? ns : 1), sizeof(double)),
           *cb = calloc((size_t)(ns > 0 ? ns : 1), sizeof(double));
    if (st == ORC_OK &&
        (!Ts || !gy || !gx || !uy || !ux || !Iw || !Pl || !P || !r || !num || !tb || !tn ||
         !Pbar || !rbar || !vx || !vy || !hb || !gb || !tmp || !Db || !Ps || !Is || !rs ||
         !ga || !In || !rsb || !uxb || !uyb || !Isb || !Psb || !mub || !Ldb || !cb))
        st = ORC_ENOMEM;
    double den = 0.0;
    for (int s = 0; st == ORC_OK && s < ns; ++s) den += ln.f[s] * ln.mu[s] * ln.mu[s];
    if (st == ORC_OK && !(den > 0.0)) st = ORC_EINVAL;

    /* forward: every iterate, by the solver itself (one iteration per call) */
    for (size_t i = 0; st == ORC_OK && i < n; ++i) Ts[i] = T0 ? T0[i] : 0.0;
    for (int it = 0; st == ORC_OK && it < n_iter; ++it) {
        memcpy(Ts + (size_t)(it + 1) * n, Ts + (size_t)it * n, sizeof(double) * n);
        st = solve_impl(ny, nx, 1, p, L, n_lines, E_keV, delta, beta, weights,
                        ORC_MODEL_NONLOCAL, D, Ts + (size_t)(it + 1) * n, 1, omega, -1.0,
                        eps_I, NULL, NULL, NULL);
    }

    /* reverse */
    for (size_t i = 0; st == ORC_OK && i < n; ++i) {
        tb[i] = Tbar_N[i];
        Db[i] = 0.0;
    }
    for (int it = n_iter - 1; st == ORC_OK && it >= 0; --it) {
        const double* T = Ts + (size_t)it * n;
        /* the forward of this iteration, recomputed */
        st = forward_impl(ny, nx, &ln, ORC_MODEL_NONLOCAL, T, P, Ps, NULL, gy, gx, uy, ux, Iw,
                          Pl);
        if (st != ORC_OK) break;
        for (size_t i = 0; i < n; ++i) {
            r[i] = D[i] - P[i];
            num[i] = 0.0;
        }
        for (int s = 0; s < ns; ++s) {
            double *I_s = Is + (size_t)s * n, *rs_s = rs + (size_t)s * n,
                   *ga_s = ga + (size_t)s * n, *In_s = In + (size_t)s * n;
            const double* P_s = Ps + (size_t)s * n;
            for (size_t i = 0; i < n; ++i) I_s[i] = ln.f[s] * exp(-ln.mu[s] * T[i]);
            if (ln.f[s] == 0.0) continue; /* a line without weight carries nothing */
            for (size_t i = 0; i < n; ++i) {
                rs_s[i] = (P[i] > 1e-30) ? r[i] * P_s[i] / P[i] : r[i] * ln.f[s];
                uy[i] = ln.c[s] * gy[i];
                ux[i] = ln.c[s] * gx[i];
            }
            orc_gather(ny, nx, rs_s, uy, ux, ga_s);
            st = filter_kind(ny, nx, p, ln.mu[s], L * ln.delta[s], 0, ga_s, tmp);
            if (st != ORC_OK) break;
            for (size_t i = 0; i < n; ++i) {
                In_s[i] = I_s[i] + omega * tmp[i];
                double fl = eps_I * ln.f[s];
                double Ic = In_s[i] < fl ? fl : In_s[i];
                num[i] += ln.f[s] * ln.mu[s] * log(Ic / ln.f[s]);
            }
        }
        if (st != ORC_OK) break;

        /* tau' = -num / den */
        double denb = 0.0;
        for (size_t i = 0; i < n; ++i) {
            denb += tb[i] * num[i] / (den * den);
            tn[i] = 0.0;
            Pbar[i] = 0.0;
            rbar[i] = 0.0;
            vx[i] = 0.0;
            vy[i] = 0.0;
        }
        for (int s = 0; s < ns; ++s) mub[s] += denb * 2.0 * ln.f[s] * ln.mu[s];
        for (int s = 0; s < ns; ++s) {
            double *rsb_s = rsb + (size_t)s * n, *uxb_s = uxb + (size_t)s * n,
                   *uyb_s = uyb + (size_t)s * n, *Isb_s = Isb + (size_t)s * n;
            for (size_t i = 0; i < n; ++i) {
                rsb_s[i] = 0.0;
                uxb_s[i] = 0.0;
                uyb_s[i] = 0.0;
                Isb_s[i] = 0.0;
            }
            if (ln.f[s] == 0.0) continue;
            const double *In_s = In + (size_t)s * n, *ga_s = ga + (size_t)s * n,
                         *rs_s = rs + (size_t)s * n;
            const double fl = eps_I * ln.f[s];
            /* num = sum_s f_s mu_s ln(I'_s / f_s), I'_s = max(I_s + omega h_s, fl) */
            for (size_t i = 0; i < n; ++i) {
                const double numb = -tb[i] / den;
                const double Ic = In_s[i] < fl ? fl : In_s[i];
                mub[s] += numb * ln.f[s] * log(Ic / ln.f[s]);
                const double Inb = In_s[i] < fl ? 0.0 : numb * ln.f[s] * ln.mu[s] / Ic;
                Isb_s[i] += Inb;
                hb[i] = omega * Inb;
            }
            /* h_s = F^-1 H_s F g_s */
            st = filter_kind(ny, nx, p, ln.mu[s], L * ln.delta[s], 0, hb, gb);
            if (st == ORC_OK) st = filter_kind(ny, nx, p, ln.mu[s], L * ln.delta[s], 1, ga_s, tmp);
            if (st != ORC_OK) break;
            for (size_t i = 0; i < n; ++i) mub[s] += hb[i] * tmp[i];
            st = filter_kind(ny, nx, p, ln.mu[s], L * ln.delta[s], 2, ga_s, tmp);
            if (st != ORC_OK) break;
            for (size_t i = 0; i < n; ++i) Ldb[s] += hb[i] * tmp[i];
            /* g_s = M_s^* r_s at the shift u_s */
            for (size_t i = 0; i < n; ++i) {
                uy[i] = ln.c[s] * gy[i];
                ux[i] = ln.c[s] * gx[i];
            }
            orc_splat(ny, nx, gb, uy, ux, rsb_s, NULL);
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(y, x);
                    double val, dux, duy;
                    interp_du(ny, nx, rs_s, y, x, uy[i], ux[i], &val, &dux, &duy);
                    uxb_s[i] += gb[i] * dux;
                    uyb_s[i] += gb[i] * duy;
                }
        }
        if (st != ORC_OK) break;
        /* r_s = r P_s / P (P > 1e-30), else r f_s */
        for (int s = 0; s < ns; ++s) {
            if (ln.f[s] == 0.0) continue;
            const double *rsb_s = rsb + (size_t)s * n, *P_s = Ps + (size_t)s * n;
            double* Psb_s = Psb + (size_t)s * n;
            for (size_t i = 0; i < n; ++i) {
                Psb_s[i] = 0.0;
                if (P[i] > 1e-30) {
                    rbar[i] += rsb_s[i] * P_s[i] / P[i];
                    Psb_s[i] += rsb_s[i] * r[i] / P[i];
                    Pbar[i] -= rsb_s[i] * r[i] * P_s[i] / (P[i] * P[i]);
                } else {
                    rbar[i] += rsb_s[i] * ln.f[s];
                }
            }
        }
        /* r = D - P, P = sum_s P_s */
        for (size_t i = 0; i < n; ++i) {
            Db[i] += rbar[i];
            Pbar[i] -= rbar[i];
        }
        for (int s = 0; s < ns; ++s) {
            if (ln.f[s] == 0.0) continue;
            double *Psb_s = Psb + (size_t)s * n, *Isb_s = Isb + (size_t)s * n,
                   *uxb_s = uxb + (size_t)s * n, *uyb_s = uyb + (size_t)s * n;
            const double* I_s = Is + (size_t)s * n;
            for (size_t i = 0; i < n; ++i) {
                Psb_s[i] += Pbar[i];
                uy[i] = ln.c[s] * gy[i];
                ux[i] = ln.c[s] * gx[i];
            }
            /* P_s = M_s[I_s] at the shift u_s */
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(y, x);
                    double val, dux, duy;
                    interp_du(ny, nx, Psb_s, y, x, uy[i], ux[i], &val, &dux, &duy);
                    Isb_s[i] += val;
                    uxb_s[i] += I_s[i] * dux;
                    uyb_s[i] += I_s[i] * duy;
                }
            /* I_s = f_s exp(-mu_s tau), u_s = c_s G[tau] */
            for (size_t i = 0; i < n; ++i) {
                tn[i] += -ln.mu[s] * I_s[i] * Isb_s[i];
                mub[s] += -T[i] * I_s[i] * Isb_s[i];
                vx[i] += ln.c[s] * uxb_s[i];
                vy[i] += ln.c[s] * uyb_s[i];
                cb[s] += uxb_s[i] * gx[i] + uyb_s[i] * gy[i];
            }
        }
        /* G^T */
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                tn[IDX(y, x)] += gT(vx + IDX(y, 0), 1, nx, x);
                tn[IDX(y, x)] += gT(vy + x, (size_t)nx, ny, y);
            }
        memcpy(tb, tn, sizeof(double) * n);
    }
    if (st == ORC_OK) {
        if (T0_bar) memcpy(T0_bar, tb, sizeof(double) * n);
        if (D_bar) memcpy(D_bar, Db, sizeof(double) * n);
        double lbar = 0.0;
        for (int s = 0; s < ns; ++s) {
            /* c_s = -L delta_s / p^2; the filter's L delta_s; mu_s = 2 k_s beta_s */
            if (delta_bar) delta_bar[s] = -L / (p * p) * cb[s] + L * Ldb[s];
            if (beta_bar) beta_bar[s] = 2.0 * ln.k[s] * mub[s];
            lbar += -ln.delta[s] / (p * p) * cb[s] + ln.delta[s] * Ldb[s];
        }
        if (L_bar) *L_bar = lbar;
    }
    free(Ts); free(gy); free(gx); free(uy); free(ux); free(Iw); free(Pl); free(P); free(r);
    free(num); free(tb); free(tn); free(Pbar); free(rbar); free(vx); free(vy); free(hb);
    free(gb); free(tmp); free(Db); free(Ps); free(Is); free(rs); free(ga); free(In);
    free(rsb); free(uxb); free(uyb); free(Isb); free(Psb); free(mub); free(Ldb); free(cb);
    lines_free(&ln);
    return st;
}

/* ------------------------------------------------------------------------ */
/* x-dependent effective spectrum ("Remark on spatially varying spectra";   */
/* Eq. 6 with db_s(x), Eq. 7 with f_s(x) and gamma_s(x); reading R13).       */
/* ------------------------------------------------------------------------ */

/* Per-column line constants from a knot table: K knot columns X_0 < ... <
 * X_{K-1} (pixel units) with, per line s and knot k, the weight w[s][k], the
 * decrement delta[s][k] and the absorption index beta[s][k].  Each is
 * interpolated linearly in the column x between knots and held constant
 * beyond the end knots.  Then, per column,
 *   f_s(x) = w_s(x) / sum_s w_s(x)            (local spectral fraction),
 *   mu_s(x) = 2 k_s beta_s(x)                 (gamma_s(x) of Eq. 7),
 *   c_s(x) = -L delta_s(x) / p^2              (shift per thickness step;
 *                                              delta_s = db_s beta_s),
 * and the preconditioner of each line takes the column means
 * mu_h[s] = mean_x mu_s(x), Ld_h[s] = L mean_x delta_s(x) (an FFT-diagonal
 * symbol needs constants).  f, mu, c are [n_lines][nx]. */
static double knot_interp(int K, const double* X, const double* v, double x)
{
    if (x <= X[0]) return v[0];
    if (x >= X[K - 1]) return v[K - 1];
    int k = 0;
    while (k + 1 < K && X[k + 1] < x) ++k;
    double t = (x - X[k]) / (X[k + 1] - X[k]);
    return v[k] + t * (v[k + 1] - v[k]);
}

int orc_xspec_params(int nx, int n_lines, const double* E_keV, int K, const double* X,
                     const double* w, const double* delta, const double* beta, double L,
                     double p, double* f, double* mu, double* c, double* mu_h, double* Ld_h)
{
    if (nx < 1 || n_lines < 1 || K < 1 || !(p > 0.0) || L < 0.0) return ORC_EINVAL;
    for (int k = 0; k + 1 < K; ++k)
        if (!(X[k + 1] > X[k])) return ORC_EINVAL;
    for (int s = 0; s < n_lines; ++s) {
        mu_h[s] = 0.0;
        Ld_h[s] = 0.0;
    }
    for (int x = 0; x < nx; ++x) {
        double wsum = 0.0;
        for (int s = 0; s < n_lines; ++s) {
            double ws = knot_interp(K, X, w + (size_t)s * K, (double)x);
            if (!(ws > 0.0)) return ORC_EINVAL;
            f[(size_t)s * nx + x] = ws;
            wsum += ws;
        }
        for (int s = 0; s < n_lines; ++s) {
            double lam = ORC_HC_EV_M / (E_keV[s] * 1e3);
            double k = 2.0 * ORC_PI / lam;
            double bs = knot_interp(K, X, beta + (size_t)s * K, (double)x);
            double ds = knot_interp(K, X, delta + (size_t)s * K, (double)x);
            f[(size_t)s * nx + x] /= wsum;
            mu[(size_t)s * nx + x] = 2.0 * k * bs;
            c[(size_t)s * nx + x] = -L * ds / (p * p);
            mu_h[s] += 2.0 * k * bs / nx;
            Ld_h[s] += L * ds / nx;
        }
    }
    return ORC_OK;
}

/* Non-local forward with per-column constants: I_s = f_s(x) exp(-mu_s(x) tau),
 * u_s = c_s(x) G[tau] (the table held constant under the derivative: the
 * spectrum varies slowly on the scale of the shift), P = sum_s M_s[I_s]. */
static void forward_x_impl(int ny, int nx, int ns, const double* f, const double* mu,
                           const double* c, const double* T, double* P, double* Ps,
                           double* dropped, const double* gy, const double* gx, double* uy,
                           double* ux, double* I, double* Pl)
{
    size_t n = (size_t)nx * (size_t)ny;
    for (size_t i = 0; i < n; ++i) P[i] = 0.0;
    for (int s = 0; s < ns; ++s) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(y, x), j = (size_t)s * nx + x;
                uy[i] = c[j] * gy[i];
                ux[i] = c[j] * gx[i];
                I[i] = f[j] * exp(-mu[j] * T[i]);
                Pl[i] = 0.0;
            }
        double lost = 0.0;
        orc_splat(ny, nx, I, uy, ux, Pl, &lost);
        for (size_t i = 0; i < n; ++i) P[i] += Pl[i];
        if (Ps) memcpy(Ps + (size_t)s * n, Pl, sizeof(double) * n);
        if (dropped) dropped[s] = lost;
    }
}

int orc_forward_x(int ny, int nx, int ns, const double* f, const double* mu, const double* c,
                  const double* T, double* P, double* Ps, double* dropped)
{
    if (ny < 2 || nx < 2 || ns < 1) return ORC_EINVAL;
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *I = alloc_n(n), *Pl = alloc_n(n);
    int st = (!gy || !gx || !uy || !ux || !I || !Pl) ? ORC_ENOMEM : ORC_OK;
    if (st == ORC_OK) {
        orc_gradient(ny, nx, T, gy, gx);
        forward_x_impl(ny, nx, ns, f, mu, c, T, P, Ps, dropped, gy, gx, uy, ux, I, Pl);
    }
    free(gy); free(gx); free(uy); free(ux); free(I); free(Pl);
    return st;
}

/* The non-local solve of "Iteration structure" with per-column constants:
 * split r_s = r P_s / P (P > 1e-30, else r f_s(x)), back-transport by the
 * gather at u_s = c_s(x) G[tau], preconditioner with the column means
 * (mu_h[s], Ld_h[s]), update I'_s = max(I_s + omega h_s, eps_I f_s(x)) and
 * the projection of Eq. 7 with per-column weights,
 *   tau' = -sum_s f_s(x) mu_s(x) ln(I'_s / f_s(x)) / sum_s f_s(x) mu_s(x)^2. */
int orc_solve_x(int ny, int nx, double p, int ns, const double* f, const double* mu,
                const double* c, const double* mu_h, const double* Ld_h, const double* D,
                double* T, int n_iter, double omega, double tol, double eps_I, double* rho,
                double* kappa, int* iters)
{
    if (ny < 2 || nx < 2 || ns < 1 || n_iter < 0) return ORC_EINVAL;
    size_t n = (size_t)nx * (size_t)ny;
    double *gy = alloc_n(n), *gx = alloc_n(n), *uy = alloc_n(n), *ux = alloc_n(n),
           *I = alloc_n(n), *Pl = alloc_n(n), *P = alloc_n(n), *r = alloc_n(n),
           *rs = alloc_n(n), *g = alloc_n(n), *num = alloc_n(n), *den = alloc_n(nx),
           *Ps = alloc_n(n * (size_t)ns);
    int st = (!gy || !gx || !uy || !ux || !I || !Pl || !P || !r || !rs || !g || !num || !den ||
              !Ps) ? ORC_ENOMEM : ORC_OK;
    for (int x = 0; st == ORC_OK && x < nx; ++x) {
        den[x] = 0.0;
        for (int s = 0; s < ns; ++s) {
            size_t j = (size_t)s * nx + x;
            den[x] += f[j] * mu[j] * mu[j];
        }
        if (!(den[x] > 0.0)) st = ORC_EINVAL;
    }
    double dnorm = 0.0;
    for (size_t i = 0; st == ORC_OK && i < n; ++i) dnorm += D[i] * D[i];
    dnorm = sqrt(dnorm);
    int it = 0;
    for (; st == ORC_OK && it < n_iter; ++it) {
        orc_gradient(ny, nx, T, gy, gx);
        forward_x_impl(ny, nx, ns, f, mu, c, T, P, Ps, NULL, gy, gx, uy, ux, I, Pl);
        double rr = 0.0;
        for (size_t i = 0; i < n; ++i) {
            r[i] = D[i] - P[i];
            rr += r[i] * r[i];
            num[i] = 0.0;
        }
        if (rho) rho[it] = dnorm > 0.0 ? sqrt(rr) / dnorm : sqrt(rr);
        for (int s = 0; s < ns; ++s) {
            const double* P_s = Ps + (size_t)s * n;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(y, x), j = (size_t)s * nx + x;
                    rs[i] = (P[i] > 1e-30) ? r[i] * P_s[i] / P[i] : r[i] * f[j];
                    uy[i] = c[j] * gy[i];
                    ux[i] = c[j] * gx[i];
                }
            orc_gather(ny, nx, rs, uy, ux, g);
            st = orc_paganin(ny, nx, p, mu_h[s], Ld_h[s], g);
            if (st != ORC_OK) break;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(y, x), j = (size_t)s * nx + x;
                    double Is = f[j] * exp(-mu[j] * T[i]);
                    double In = Is + omega * g[i];
                    double fl = eps_I * f[j];
                    if (In < fl) In = fl;
                    num[i] += f[j] * mu[j] * log(In / f[j]);
                }
        }
        if (st != ORC_OK) break;
        double dd = 0.0, tt = 0.0;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(y, x);
                double tn = -num[i] / den[x];
                dd += (tn - T[i]) * (tn - T[i]);
                tt += tn * tn;
                T[i] = tn;
            }
        double kap = tt > 0.0 ? sqrt(dd / tt) : sqrt(dd);
        if (kappa) kappa[it] = kap;
        if (kap <= tol) {
            ++it;
            break;
        }
    }
    if (iters) *iters = it;
    free(gy); free(gx); free(uy); free(ux); free(I); free(Pl); free(P); free(r); free(rs);
    free(g); free(num); free(den); free(Ps);
    return st;
}
