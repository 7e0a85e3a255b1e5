/*
 * FP64 CPU oracle for TV-regularised multi-coil MRI reconstruction with ADMM
 * (Lu et al., "Accelerating MRI Reconstruction on TPUs", arXiv 2006.14080).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may call, link or
 * include this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Plain, slow, obviously correct: every operator is its definition written out
 * as a direct sum in double precision.  OpenMP only splits independent outputs
 * across threads; the order of every individual sum is the textbook one.
 *
 * Conventions (readings of the paper where it is silent):
 *   - image x is [nx][ny] complex, pixel coordinates x_i = i - nx/2 (integer
 *     division), y_j = j - ny/2; trajectory k is [nk][2] in cycles/pixel.
 *   - the DFT is unnormalised, sign -i forward, +i adjoint (Eq. 1).
 *   - Theta is the pair of forward differences with zero padding past the last
 *     pixel, stacked as [2][nx][ny] (x-differences then y-differences).
 *   - soft threshold is the complex-magnitude shrink with threshold lambda/beta
 *     (Eq. 8-9; reduces to Eq. 9 for real input).
 *   - CG starts from r = b - A x0 (Alg. 2), dot products are sum conj(u) v
 *     and alpha uses the real part.
 *   - ADMM starts from x = 0, eta = 0; CG warm-starts from the current x; the
 *     dual update uses the new image (Eq. 8, third line).
 * Arrays are interleaved complex (re, im) doubles.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct { double re, im; } cpx;

static inline cpx cmul(cpx a, cpx b) { cpx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cpx cconj(cpx a) { cpx r = {a.re, -a.im}; return r; }
static inline cpx cadd(cpx a, cpx b) { cpx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cpx csub(cpx a, cpx b) { cpx r = {a.re - b.re, a.im - b.im}; return r; }
static inline cpx cscale(cpx a, double s) { cpx r = {a.re * s, a.im * s}; return r; }
static inline double cabs2(cpx a) { return a.re * a.re + a.im * a.im; }

/* exp(-i 2 pi t): the phase is reduced to its fractional part first so that
 * the argument of sin/cos stays in [-pi, pi]. */
static inline cpx phasor_fwd(double t) {
    double f = t - rint(t);
    cpx r = {cos(2.0 * M_PI * f), -sin(2.0 * M_PI * f)};
    return r;
}

static inline double coord(int i, int n) { return (double)(i - n / 2); }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 1-2: d[c][kappa] = sum_n s[c][n] x[n] exp(-i 2 pi k_kappa . r_n).
 * Direct summation over all pixels; one phasor per (kappa, pixel) is shared
 * by the coils. */
void orc_forward(int nx, int ny, int nk, int nc, const double *traj,
                 const double *image, const double *maps, double *kspace) {
    const cpx *x = (const cpx *)image;
    const cpx *s = (const cpx *)maps;
    cpx *d = (cpx *)kspace;
    const int npix = nx * ny;
    cpx *sx = (cpx *)malloc(sizeof(cpx) * (size_t)nc * npix);
    for (int c = 0; c < nc; ++c)
        for (int n = 0; n < npix; ++n) sx[(size_t)c * npix + n] = cmul(s[(size_t)c * npix + n], x[n]);
#pragma omp parallel
    {
        cpx *acc = (cpx *)malloc(sizeof(cpx) * (size_t)nc);
#pragma omp for schedule(static)
        for (int kk = 0; kk < nk; ++kk) {
            const double kx = traj[2 * kk], ky = traj[2 * kk + 1];
            for (int c = 0; c < nc; ++c) { acc[c].re = 0.0; acc[c].im = 0.0; }
            for (int i = 0; i < nx; ++i) {
                for (int j = 0; j < ny; ++j) {
                    cpx e = phasor_fwd(kx * coord(i, nx) + ky * coord(j, ny));
                    int n = i * ny + j;
                    for (int c = 0; c < nc; ++c) acc[c] = cadd(acc[c], cmul(sx[(size_t)c * npix + n], e));
                }
            }
            for (int c = 0; c < nc; ++c) d[(size_t)c * nk + kk] = acc[c];
        }
        free(acc);
    }
    free(sx);
}

/* Adjoint of Eq. 1: x[n] = sum_c conj(s[c][n]) sum_kappa d[c][kappa] exp(+i 2 pi k_kappa . r_n). */
void orc_adjoint(int nx, int ny, int nk, int nc, const double *traj,
                 const double *kspace, const double *maps, double *image) {
    const cpx *d = (const cpx *)kspace;
    const cpx *s = (const cpx *)maps;
    cpx *x = (cpx *)image;
    const int npix = nx * ny;
#pragma omp parallel
    {
        cpx *acc = (cpx *)malloc(sizeof(cpx) * (size_t)nc);
#pragma omp for schedule(static)
        for (int n = 0; n < npix; ++n) {
            const int i = n / ny, j = n % ny;
            for (int c = 0; c < nc; ++c) { acc[c].re = 0.0; acc[c].im = 0.0; }
            for (int kk = 0; kk < nk; ++kk) {
                cpx e = cconj(phasor_fwd(traj[2 * kk] * coord(i, nx) + traj[2 * kk + 1] * coord(j, ny)));
                for (int c = 0; c < nc; ++c) acc[c] = cadd(acc[c], cmul(d[(size_t)c * nk + kk], e));
            }
            cpx out = {0.0, 0.0};
            for (int c = 0; c < nc; ++c) out = cadd(out, cmul(cconj(s[(size_t)c * npix + n]), acc[c]));
            x[n] = out;
        }
        free(acc);
    }
}

/* The adjoint of Eq. 1 evaluated only at the npick pixels listed in pix
 * (flat indices i*ny + j); out[q] receives the value at pix[q].  Same sum as
 * orc_adjoint, for spot checks of large problems. */
void orc_adjoint_at(int nx, int ny, int nk, int nc, const double *traj, const double *kspace,
                    const double *maps, int npick, const int *pix, double *out) {
    const cpx *d = (const cpx *)kspace;
    const cpx *s = (const cpx *)maps;
    cpx *x = (cpx *)out;
    const int npix = nx * ny;
#pragma omp parallel
    {
        cpx *acc = (cpx *)malloc(sizeof(cpx) * (size_t)nc);
#pragma omp for schedule(static)
        for (int q = 0; q < npick; ++q) {
            const int n = pix[q], i = n / ny, j = n % ny;
            for (int c = 0; c < nc; ++c) { acc[c].re = 0.0; acc[c].im = 0.0; }
            for (int kk = 0; kk < nk; ++kk) {
                cpx e = cconj(phasor_fwd(traj[2 * kk] * coord(i, nx) + traj[2 * kk + 1] * coord(j, ny)));
                for (int c = 0; c < nc; ++c) acc[c] = cadd(acc[c], cmul(d[(size_t)c * nk + kk], e));
            }
            cpx o = {0.0, 0.0};
            for (int c = 0; c < nc; ++c) o = cadd(o, cmul(cconj(s[(size_t)c * npix + n]), acc[c]));
            x[q] = o;
        }
        free(acc);
    }
}

/* Theta: first-order forward differences along each axis (conv1d with kernel
 * [-1, 1], zero padding past the last pixel).  g is [2][nx][ny]. */
void orc_tv_forward(int nx, int ny, const double *image, double *grad) {
    const cpx *x = (const cpx *)image;
    cpx *g = (cpx *)grad;
    const cpx zero = {0.0, 0.0};
    const int npix = nx * ny;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j) {
            cpx xn = x[i * ny + j];
            cpx xi = (i + 1 < nx) ? x[(i + 1) * ny + j] : zero;
            cpx xj = (j + 1 < ny) ? x[i * ny + j + 1] : zero;
            g[i * ny + j] = csub(xi, xn);
            g[npix + i * ny + j] = csub(xj, xn);
        }
}

/* Theta^H, the exact transpose of orc_tv_forward:
 * x[i][j] = (g0[i-1][j] - g0[i][j]) + (g1[i][j-1] - g1[i][j]), g[-1] = 0. */
void orc_tv_adjoint(int nx, int ny, const double *grad, double *image) {
    const cpx *g = (const cpx *)grad;
    cpx *x = (cpx *)image;
    const cpx zero = {0.0, 0.0};
    const int npix = nx * ny;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j) {
            cpx a = (i > 0) ? g[(i - 1) * ny + j] : zero;
            cpx b = (j > 0) ? g[npix + i * ny + j - 1] : zero;
            cpx v = csub(a, g[i * ny + j]);
            v = cadd(v, csub(b, g[npix + i * ny + j]));
            x[i * ny + j] = v;
        }
}

/* Eq. 9 for complex input: S_t(a) = a (1 - t/|a|) if |a| > t, else 0. */
void orc_shrink(int n, double t, const double *in, double *out) {
    const cpx *a = (const cpx *)in;
    cpx *m = (cpx *)out;
    for (int q = 0; q < n; ++q) {
        double mag = sqrt(cabs2(a[q]));
        if (mag <= t) { m[q].re = 0.0; m[q].im = 0.0; }
        else m[q] = cscale(a[q], 1.0 - t / mag);
    }
}

/* Eq. 11: A p = F^H F p + (beta/2) Theta^H Theta p. */
void orc_normal(int nx, int ny, int nk, int nc, const double *traj, const double *maps,
                double beta, const double *p, double *out) {
    const int npix = nx * ny;
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)nc * nk);
    double *g = (double *)malloc(sizeof(double) * 4 * (size_t)npix);
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)npix);
    orc_forward(nx, ny, nk, nc, traj, p, maps, y);
    orc_adjoint(nx, ny, nk, nc, traj, y, maps, out);
    orc_tv_forward(nx, ny, p, g);
    orc_tv_adjoint(nx, ny, g, t);
    for (int q = 0; q < 2 * npix; ++q) out[q] += 0.5 * beta * t[q];
    free(y); free(g); free(t);
}

static double dot_re(int n, const cpx *u, const cpx *v) {
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += u[q].re * v[q].re + u[q].im * v[q].im;  /* Re(conj(u) v) */
    return s;
}

/* Alg. 2: conjugate gradient on A x = b from x0 (in/out in x), at most
 * max_iter steps, stopping when tau = ||r||^2 <= atol^2.  tau_hist (nullable,
 * length max_iter + 1) receives tau before each step and after the last.
 * Returns the number of steps taken. */
int orc_cg(int nx, int ny, int nk, int nc, const double *traj, const double *maps, double beta,
           const double *b, double *x, int max_iter, double atol, double *tau_hist) {
    const int npix = nx * ny;
    cpx *r = (cpx *)malloc(sizeof(cpx) * npix);
    cpx *d = (cpx *)malloc(sizeof(cpx) * npix);
    cpx *ad = (cpx *)malloc(sizeof(cpx) * npix);
    cpx *xv = (cpx *)x;
    const cpx *bv = (const cpx *)b;
    orc_normal(nx, ny, nk, nc, traj, maps, beta, x, (double *)ad);
    for (int q = 0; q < npix; ++q) { r[q] = csub(bv[q], ad[q]); d[q] = r[q]; }
    double tau = dot_re(npix, r, r);
    int it = 0;
    if (tau_hist) tau_hist[0] = tau;
    while (it < max_iter && tau > atol * atol) {
        orc_normal(nx, ny, nk, nc, traj, maps, beta, (const double *)d, (double *)ad);
        double alpha = tau / dot_re(npix, d, ad);
        for (int q = 0; q < npix; ++q) {
            xv[q] = cadd(xv[q], cscale(d[q], alpha));
            r[q] = csub(r[q], cscale(ad[q], alpha));
        }
        double tau_next = dot_re(npix, r, r);
        double bcg = tau_next / tau;
        for (int q = 0; q < npix; ++q) d[q] = cadd(r[q], cscale(d[q], bcg));
        tau = tau_next;
        ++it;
        if (tau_hist) tau_hist[it] = tau;
    }
    free(r); free(d); free(ad);
    return it;
}

/* Eq. 3: f(x) = ||F x - d||^2 + lambda * sum |Theta x| (complex modulus,
 * summed over both difference fields). */
double orc_objective(int nx, int ny, int nk, int nc, const double *traj, const double *maps,
                     const double *kspace, double lambda, const double *image) {
    const int npix = nx * ny;
    cpx *y = (cpx *)malloc(sizeof(cpx) * (size_t)nc * nk);
    cpx *g = (cpx *)malloc(sizeof(cpx) * 2 * (size_t)npix);
    const cpx *d = (const cpx *)kspace;
    orc_forward(nx, ny, nk, nc, traj, image, maps, (double *)y);
    double fid = 0.0;
    for (size_t q = 0; q < (size_t)nc * nk; ++q) fid += cabs2(csub(y[q], d[q]));
    orc_tv_forward(nx, ny, image, (double *)g);
    double l1 = 0.0;
    for (int q = 0; q < 2 * npix; ++q) l1 += sqrt(cabs2(g[q]));
    free(y); free(g);
    return fid + lambda * l1;
}

/* Alg. 4 with Eq. 6-12:
 *   x = 0, eta = 0
 *   repeat (at most admm_iters times, while alpha > rtol^2):
 *     mu    = S_{lambda/beta}(Theta x + eta)                       (Eq. 8)
 *     b     = F^H d + (beta/2) Theta^H (mu - eta)                  (Eq. 12)
 *     x'    = CG(A, b, x0 = x, cg_iters, atol)                     (Eq. 10-11, Alg. 2)
 *     alpha = ||x' - x||^2 / ||x'||^2                              (Alg. 4)
 *     eta   = eta + Theta x' - mu                                  (Eq. 8, dual)
 *     x     = x'
 * Outputs the final image; obj_hist / alpha_hist (nullable, length
 * admm_iters) receive f(x') and alpha after each outer step.  mu_out and
 * eta_out (nullable, [2][nx][ny]) receive the final auxiliary and dual
 * variables.  Returns the number of outer steps taken. */
int orc_admm(int nx, int ny, int nk, int nc, const double *traj, const double *maps,
             const double *kspace, double lambda, double beta, int admm_iters, int cg_iters,
             double rtol, double atol, double *image_out, double *obj_hist, double *alpha_hist,
             double *mu_out, double *eta_out) {
    const int npix = nx * ny;
    cpx *x = (cpx *)image_out;
    cpx *xn = (cpx *)malloc(sizeof(cpx) * npix);
    cpx *fhd = (cpx *)malloc(sizeof(cpx) * npix);
    cpx *eta = (cpx *)calloc(2 * (size_t)npix, sizeof(cpx));
    cpx *mu = (cpx *)calloc(2 * (size_t)npix, sizeof(cpx));
    cpx *t = (cpx *)malloc(sizeof(cpx) * 2 * (size_t)npix);
    cpx *b = (cpx *)malloc(sizeof(cpx) * npix);
    memset(x, 0, sizeof(cpx) * npix);
    orc_adjoint(nx, ny, nk, nc, traj, kspace, maps, (double *)fhd);
    double alpha = 1.0;
    int m = 0;
    while (m < admm_iters && alpha > rtol * rtol) {
        /* mu-update */
        orc_tv_forward(nx, ny, (const double *)x, (double *)t);
        for (int q = 0; q < 2 * npix; ++q) t[q] = cadd(t[q], eta[q]);
        orc_shrink(2 * npix, lambda / beta, (const double *)t, (double *)mu);
        /* right-hand side */
        for (int q = 0; q < 2 * npix; ++q) t[q] = csub(mu[q], eta[q]);
        orc_tv_adjoint(nx, ny, (const double *)t, (double *)b);
        for (int q = 0; q < npix; ++q) b[q] = cadd(fhd[q], cscale(b[q], 0.5 * beta));
        /* primal update by CG, warm-started from x */
        memcpy(xn, x, sizeof(cpx) * npix);
        orc_cg(nx, ny, nk, nc, traj, maps, beta, (const double *)b, (double *)xn, cg_iters, atol, NULL);
        /* relative change */
        double num = 0.0, den = 0.0;
        for (int q = 0; q < npix; ++q) { num += cabs2(csub(xn[q], x[q])); den += cabs2(xn[q]); }
        alpha = num / (den > 1e-300 ? den : 1e-300);
        /* dual update with the new image */
        orc_tv_forward(nx, ny, (const double *)xn, (double *)t);
        for (int q = 0; q < 2 * npix; ++q) eta[q] = csub(cadd(eta[q], t[q]), mu[q]);
        memcpy(x, xn, sizeof(cpx) * npix);
        if (obj_hist) obj_hist[m] = orc_objective(nx, ny, nk, nc, traj, maps, kspace, lambda, (const double *)x);
        if (alpha_hist) alpha_hist[m] = alpha;
        ++m;
    }
    if (mu_out) memcpy(mu_out, mu, sizeof(cpx) * 2 * (size_t)npix);
    if (eta_out) memcpy(eta_out, eta, sizeof(cpx) * 2 * (size_t)npix);
    free(xn); free(fhd); free(eta); free(mu); free(t); free(b);
    return m;
}
