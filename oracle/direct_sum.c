/*
 * Oracle: plain FP64 direct summation of an oscillatory integral operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only tests/, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py use it.  It shares no code with the CUDA library.
 *
 * What it computes (paper Sec. 3.2, contraction G = K x_{d+1..2d} F of Alg. 2,
 * written out as the plain definition, without any compression):
 *
 *   forward  u(x^i) = sum_j K(x^i, y^j) f(y^j)              for each RHS v
 *   adjoint  v(y^j) = sum_i conj(K(x^i, y^j)) g(x^i)        for each RHS v
 *
 * on tensor grids x^i = (x_1[i_1], ..., x_d[i_d]), y^j = (y_1[j_1], ..., y_d[j_d]).
 * Arrays are complex128 stored as interleaved (re, im) doubles in C order over
 * (n_1, ..., n_d, nv): the RHS index is innermost.  Output rows (or columns for
 * the adjoint) are given as flat C-order indices so that large operators can be
 * checked on a sample of outputs.
 *
 * Kernels (all evaluated in FP64 with libm, no range reduction):
 *   1 Fourier   K = exp(-2 pi i x.y)                       (Sec. 4.3, sign as configured)
 *   2 Helmholtz K = exp(i kappa rho) / rho,               (Sec. 4.1, outgoing sign as configured)
 *               rho = sqrt(|x - y|^2 + h^2), par = (kappa, h): h is the distance
 *               between the two grids along an axis outside the d grid axes
 *               (h = 0: cubes; d = 2, h = 1: the parallel plates of Sec. 4.1)
 *   3 Radon     K = exp(2 pi i (x.xi + c(x)|xi|)),
 *               c(x) = a + b prod_k sin(2 pi x_k)          (Sec. 4.2, Eq. randon3d form)
 *   4 Radon, anisotropic (d = 2, Sec. 4.2 Eq. randon2d):
 *               K = exp(2 pi i (x.xi + sqrt(c1^2 xi_1^2 + c2^2 xi_2^2))),
 *               c1 = a1 + b1 sin(2 pi x_1) sin(2 pi x_2), c2 = a2 + b2 cos(2 pi x_1) cos(2 pi x_2),
 *               par = (a1, b1, a2, b2)
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TBO_MAX_D 8

static const double TWO_PI = 6.283185307179586476925286766559;

/* One kernel entry K(x, y) for points x, y in R^d. */
static double complex tbo_entry(int kind, const double *par, int d,
                                const double *x, const double *y)
{
    if (kind == 1) {
        double p = 0.0;
        for (int k = 0; k < d; ++k) p += x[k] * y[k];
        return cexp(-I * TWO_PI * p);
    }
    if (kind == 2) {
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = x[k] - y[k];
            r2 += t * t;
        }
        double rho = sqrt(r2 + par[1] * par[1]);
        return cexp(I * par[0] * rho) / rho;
    }
    if (kind == 4) {
        if (d != 2) return 0.0;
        double c1 = par[0] + par[1] * sin(TWO_PI * x[0]) * sin(TWO_PI * x[1]);
        double c2 = par[2] + par[3] * cos(TWO_PI * x[0]) * cos(TWO_PI * x[1]);
        double phi = x[0] * y[0] + x[1] * y[1] + sqrt(c1 * c1 * y[0] * y[0] + c2 * c2 * y[1] * y[1]);
        return cexp(I * TWO_PI * phi);
    }
    if (kind == 3) {
        double xy = 0.0, yy = 0.0, s = 1.0;
        for (int k = 0; k < d; ++k) {
            xy += x[k] * y[k];
            yy += y[k] * y[k];
            s *= sin(TWO_PI * x[k]);
        }
        double c = par[0] + par[1] * s;
        return cexp(I * TWO_PI * (xy + c * sqrt(yy)));
    }
    return 0.0;
}

static void tbo_point(int d, const int64_t *sizes, const double *coords,
                      int64_t flat, double *pt)
{
    /* coords: axis k occupies coords[off_k .. off_k + sizes[k]) */
    int64_t idx[TBO_MAX_D];
    for (int k = d - 1; k >= 0; --k) {
        idx[k] = flat % sizes[k];
        flat /= sizes[k];
    }
    int64_t off = 0;
    for (int k = 0; k < d; ++k) {
        pt[k] = coords[off + idx[k]];
        off += sizes[k];
    }
}

int tbo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Single entry K(x, y) written to out[0..1] as (re, im). */
int tbo_kernel_entry(int kind, const double *par, int d, const double *x,
                     const double *y, double *out)
{
    if (d < 1 || d > TBO_MAX_D) return -1;
    double complex k = tbo_entry(kind, par, d, x, y);
    out[0] = creal(k);
    out[1] = cimag(k);
    return 0;
}

/*
 * Forward direct sum on selected output rows.
 *   m[d], xc: target grid sizes and concatenated per-axis coordinates
 *   n[d], yc: source grid sizes and coordinates
 *   f: (prod n, nv) complex interleaved;  rows[nrows]: flat target indices
 *   out: (nrows, nv) complex interleaved
 */
int tbo_apply(int kind, const double *par, int d,
              const int64_t *m, const double *xc,
              const int64_t *n, const double *yc,
              const double *f, int64_t nv,
              const int64_t *rows, int64_t nrows, double *out)
{
    if (d < 1 || d > TBO_MAX_D || nv < 1) return -1;
    int64_t N = 1;
    for (int k = 0; k < d; ++k) N *= n[k];

#pragma omp parallel
    {
        double complex *acc = (double complex *)malloc(sizeof(double complex) * nv);
        double x[TBO_MAX_D], y[TBO_MAX_D];
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            tbo_point(d, m, xc, rows[r], x);
            for (int64_t v = 0; v < nv; ++v) acc[v] = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                tbo_point(d, n, yc, j, y);
                double complex kv = tbo_entry(kind, par, d, x, y);
                const double *fj = f + 2 * j * nv;
                for (int64_t v = 0; v < nv; ++v)
                    acc[v] += kv * (fj[2 * v] + I * fj[2 * v + 1]);
            }
            for (int64_t v = 0; v < nv; ++v) {
                out[2 * (r * nv + v)] = creal(acc[v]);
                out[2 * (r * nv + v) + 1] = cimag(acc[v]);
            }
        }
        free(acc);
    }
    return 0;
}

/*
 * Adjoint direct sum on selected output columns (source points):
 *   out[c, v] = sum_i conj(K(x^i, y^{cols[c]})) g[i, v]
 */
int tbo_apply_adjoint(int kind, const double *par, int d,
                      const int64_t *m, const double *xc,
                      const int64_t *n, const double *yc,
                      const double *g, int64_t nv,
                      const int64_t *cols, int64_t ncols, double *out)
{
    if (d < 1 || d > TBO_MAX_D || nv < 1) return -1;
    int64_t M = 1;
    for (int k = 0; k < d; ++k) M *= m[k];

#pragma omp parallel
    {
        double complex *acc = (double complex *)malloc(sizeof(double complex) * nv);
        double x[TBO_MAX_D], y[TBO_MAX_D];
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < ncols; ++c) {
            tbo_point(d, n, yc, cols[c], y);
            for (int64_t v = 0; v < nv; ++v) acc[v] = 0.0;
            for (int64_t i = 0; i < M; ++i) {
                tbo_point(d, m, xc, i, x);
                double complex kv = conj(tbo_entry(kind, par, d, x, y));
                const double *gi = g + 2 * i * nv;
                for (int64_t v = 0; v < nv; ++v)
                    acc[v] += kv * (gi[2 * v] + I * gi[2 * v + 1]);
            }
            for (int64_t v = 0; v < nv; ++v) {
                out[2 * (c * nv + v)] = creal(acc[v]);
                out[2 * (c * nv + v) + 1] = cimag(acc[v]);
            }
        }
        free(acc);
    }
    return 0;
}
