/*
 * oracle.c — FP64 CPU oracle for the paper's FFT -> filter -> IFFT path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA library; the two are compared against each other.
 *
 * Every routine is a plain, slow, obviously correct restatement of a
 * definition or algorithm of Higuera, Sarria, Fonseca and Idarraga,
 * "Construction of an algorithm in parallel for the Fast Fourier Transform"
 * (arXiv cs/0103001), evaluated in IEEE double precision:
 *
 *   orc_dft          Eq. E2 / Eq. coefFourier, written out as the O(N^2) sum
 *   orc_idft         Eq. E3 evaluated at x_j = 2*pi*j/N (unscaled)
 *   orc_dft_bins     Eq. E2 for a chosen list of output bins, O(N) per bin
 *   orc_fft          Sec. 2 radix-2 "interpolation tree" (decimation in time,
 *                    leaves in bit-reversed order), 1/N applied once at the end
 *   orc_ifft         Sec. 3: the inverse as N * FFT read in reverse order
 *   orc_fft2/ifft2   Sec. 4: row transforms, then column transforms
 *                    (per-axis convention, or Eq. 5 with its "x M" step)
 *   orc_pipeline     Sec. 5: fft2 -> multiply Re and Im by a real filter ->
 *                    ifft2 -> real part
 *   orc_pipeline_grad  gradients of the Sec. 5 pipeline (closed forms)
 *
 * Complex arrays are interleaved (re, im) doubles.  Every function returns 0
 * on success and a negative number on a bad argument.  None of them has a
 * tolerance: pins in the test-suite check them against closed forms,
 * invariants, brute force and numpy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* Table 2's vector Z: Z_j = exp(-2*pi*i*j/N), j = 0..N-1, in FP64.  The
 * phase index is an exact integer, so no angle is reduced in floating point. */
static double *make_Z(int64_t n) {
    double *z = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!z) return NULL;
    for (int64_t j = 0; j < n; ++j) {
        double a = 2.0 * ORC_PI * (double)j / (double)n;
        z[2 * j] = cos(a);
        z[2 * j + 1] = -sin(a);
    }
    return z;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Eq. E2 (and Eq. coefFourier): c_k = (1/N) sum_j f_j exp(-2 pi i k j / N).
 * Eq. E3 at x_j = 2 pi j / N:   f_j = sum_k c_k exp(+i k x_j), no scale.
 * The exponent index (k*j mod N) is reduced in exact integer arithmetic.
 * Any N >= 1 is accepted here (the definition does not need a power of two).
 * ------------------------------------------------------------------------- */
static void dft_one(const double *x, double *y, int64_t n, int inverse, const double *Z) {
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t p = (k * j) % n;
            double wr = Z[2 * p], wi = inverse ? -Z[2 * p + 1] : Z[2 * p + 1];
            double xr = x[2 * j], xi = x[2 * j + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        if (!inverse) {
            sr /= (double)n;
            si /= (double)n;
        }
        y[2 * k] = sr;
        y[2 * k + 1] = si;
    }
}

static int dft_batch(const double *x, double *y, int64_t n, int64_t batch, int inverse) {
    if (!x || !y || n < 1 || batch < 0) return -1;
    double *Z = make_Z(n);
    if (!Z) return -2;
    int64_t b;
#pragma omp parallel for schedule(dynamic)
    for (b = 0; b < batch; ++b) dft_one(x + 2 * b * n, y + 2 * b * n, n, inverse, Z);
    free(Z);
    return 0;
}

int orc_dft(const double *x, double *y, int64_t n, int64_t batch) { return dft_batch(x, y, n, batch, 0); }
int orc_idft(const double *x, double *y, int64_t n, int64_t batch) { return dft_batch(x, y, n, batch, 1); }

/* Eq. E2 (inverse = 0) or Eq. E3 (inverse = 1) for the listed output bins of
 * ONE transform of length n: y[i] = value at bin bins[i].  O(n) per bin. */
int orc_dft_bins(const double *x, int64_t n, const int64_t *bins, int64_t nbins, int inverse, double *y) {
    if (!x || !y || !bins || n < 1 || nbins < 0) return -1;
    double *Z = make_Z(n);
    if (!Z) return -2;
    int64_t i;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (i = 0; i < nbins; ++i) {
        int64_t k = bins[i];
        if (k < 0 || k >= n) {
            bad = 1;
            continue;
        }
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t p = (k * j) % n;
            double wr = Z[2 * p], wi = inverse ? -Z[2 * p + 1] : Z[2 * p + 1];
            sr += x[2 * j] * wr - x[2 * j + 1] * wi;
            si += x[2 * j] * wi + x[2 * j + 1] * wr;
        }
        if (!inverse) {
            sr /= (double)n;
            si /= (double)n;
        }
        y[2 * i] = sr;
        y[2 * i + 1] = si;
    }
    free(Z);
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Sec. 2, the "interpolation tree": radix-2 decimation in time.  A node at
 * level n merges the two length-2^(n-1) transforms of its children, the child
 * built from the even-indexed samples and the child built from the odd ones,
 * so that the leaves of the tree, read left to right, are the samples in
 * bit-reversed order (C(0), C(4), C(2), C(6), C(1), C(5), C(3), C(7) for N=8).
 * The merge factor of a length-L node is exp(-2 pi i k / L) = Z[k * N / L].
 * Each level costs N products, so the tree costs N log2 N.
 *
 * tree(x, s, L, y): y[0..L) = unscaled DFT of x[0], x[s], ..., x[(L-1)s].
 * ------------------------------------------------------------------------- */
static void tree(const double *x, int64_t s, int64_t L, double *y, const double *Z, int64_t zstep) {
    if (L == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    int64_t h = L / 2;
    tree(x, 2 * s, h, y, Z, 2 * zstep);                /* even samples -> y[0..h)  */
    tree(x + 2 * s, 2 * s, h, y + 2 * h, Z, 2 * zstep); /* odd samples  -> y[h..L) */
    for (int64_t k = 0; k < h; ++k) {
        double wr = Z[2 * k * zstep], wi = Z[2 * k * zstep + 1];
        double er = y[2 * k], ei = y[2 * k + 1];
        double or_ = y[2 * (k + h)], oi = y[2 * (k + h) + 1];
        double tr = or_ * wr - oi * wi, ti = or_ * wi + oi * wr;
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (k + h)] = er - tr;
        y[2 * (k + h) + 1] = ei - ti;
    }
}

/* Sec. 2 FFT with the Eq. E2 normalisation: the tree, then 1/N once. */
static int fft_one(const double *x, double *y, int64_t n, const double *Z) {
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!tmp) return -2;
    tree(x, 1, n, tmp, Z, 1);
    for (int64_t k = 0; k < 2 * n; ++k) y[k] = tmp[k] / (double)n;
    free(tmp);
    return 0;
}

/* Sec. 3: the inverse transform through the forward one.  Evaluating the
 * exponential polynomial p at 2*pi - x_k turns the inverse sum into a forward
 * sum, so f_k = p(x_k) = N * FFT(c)[(N - k) mod N]: the forward FFT times N,
 * read in reverse order (index 0 stays in place because p(2*pi) = p(0)). */
static int ifft_one(const double *c, double *f, int64_t n, const double *Z) {
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!t) return -2;
    int rc = fft_one(c, t, n, Z);
    if (!rc)
        for (int64_t k = 0; k < n; ++k) {
            int64_t r = (n - k) % n;
            f[2 * k] = (double)n * t[2 * r];
            f[2 * k + 1] = (double)n * t[2 * r + 1];
        }
    free(t);
    return rc;
}

/* n must be 2^m with m >= 1 (Sec. 3, complexity section). */
static int fft_many(const double *x, double *y, int64_t n, int64_t batch, int inverse) {
    if (!x || !y || batch < 0 || n < 2 || !is_pow2(n)) return -1;
    double *Z = make_Z(n);
    if (!Z) return -2;
    int64_t b;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (b = 0; b < batch; ++b) {
        int rc = inverse ? ifft_one(x + 2 * b * n, y + 2 * b * n, n, Z) : fft_one(x + 2 * b * n, y + 2 * b * n, n, Z);
        if (rc) bad = 1;
    }
    free(Z);
    return bad ? -2 : 0;
}

int orc_fft(const double *x, double *y, int64_t n, int64_t batch) { return fft_many(x, y, n, batch, 0); }
int orc_ifft(const double *c, double *f, int64_t n, int64_t batch) { return fft_many(c, f, n, batch, 1); }

/* ---------------------------------------------------------------------------
 * Sec. 4, two-dimensional transform of an N x M array (N rows indexed by x,
 * M columns indexed by y; row-major, so a row is contiguous).
 *
 * conv = 0 (per-axis): the 1D definition on each axis, i.e. 1/M on the rows
 *   and 1/N on the columns: F = (1/(N M)) sum_x sum_y f exp(-i 2 pi (ux/N + vy/M)).
 * conv = 1 (Eq. 5): F(u,v) = (1/N) sum sum f exp(...), built the paper's way:
 *   "FFT on rows -> multiplication by M -> FFT on columns".  Eq. 5's F is M
 *   times the per-axis F.
 * The inverse undoes the forward of the same convention: per-axis applies
 * Eq. E3 on each axis (no scale); Eq. 5's 2D-IDFT has 1/M in front.
 * ------------------------------------------------------------------------- */
static int columns_1d(double *a, int64_t rows, int64_t cols, int inverse) {
    double *Z = make_Z(rows);
    if (!Z) return -2;
    int64_t c;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (c = 0; c < cols; ++c) {
        double *col = (double *)malloc(sizeof(double) * 2 * (size_t)rows);
        double *out = (double *)malloc(sizeof(double) * 2 * (size_t)rows);
        if (!col || !out) {
            bad = 1;
            free(col);
            free(out);
            continue;
        }
        for (int64_t r = 0; r < rows; ++r) {
            col[2 * r] = a[2 * (r * cols + c)];
            col[2 * r + 1] = a[2 * (r * cols + c) + 1];
        }
        if ((inverse ? ifft_one(col, out, rows, Z) : fft_one(col, out, rows, Z)) != 0) bad = 1;
        for (int64_t r = 0; r < rows; ++r) {
            a[2 * (r * cols + c)] = out[2 * r];
            a[2 * (r * cols + c) + 1] = out[2 * r + 1];
        }
        free(col);
        free(out);
    }
    free(Z);
    return bad ? -2 : 0;
}

int orc_fft2(const double *x, double *y, int64_t rows, int64_t cols, int64_t batch, int conv) {
    if (!x || !y || batch < 0 || rows < 2 || cols < 2 || !is_pow2(rows) || !is_pow2(cols)) return -1;
    if (conv != 0 && conv != 1) return -1;
    for (int64_t b = 0; b < batch; ++b) {
        const double *xb = x + 2 * b * rows * cols;
        double *yb = y + 2 * b * rows * cols;
        int rc = orc_fft(xb, yb, cols, rows); /* FFT on rows */
        if (rc) return rc;
        if (conv == 1) /* multiplication by M */
            for (int64_t i = 0; i < 2 * rows * cols; ++i) yb[i] *= (double)cols;
        rc = columns_1d(yb, rows, cols, 0); /* FFT on columns */
        if (rc) return rc;
    }
    return 0;
}

int orc_ifft2(const double *x, double *y, int64_t rows, int64_t cols, int64_t batch, int conv) {
    if (!x || !y || batch < 0 || rows < 2 || cols < 2 || !is_pow2(rows) || !is_pow2(cols)) return -1;
    if (conv != 0 && conv != 1) return -1;
    for (int64_t b = 0; b < batch; ++b) {
        const double *xb = x + 2 * b * rows * cols;
        double *yb = y + 2 * b * rows * cols;
        int rc = orc_ifft(xb, yb, cols, rows);
        if (rc) return rc;
        rc = columns_1d(yb, rows, cols, 1);
        if (rc) return rc;
        if (conv == 1)
            for (int64_t i = 0; i < 2 * rows * cols; ++i) yb[i] /= (double)cols;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Sec. 5, the application: transform the image, multiply the real and the
 * imaginary part of every frequency (u,v) by the real filter value H(u,v),
 * transform back, keep the real part as the filtered image.
 *   img : batch x rows x cols real
 *   H   : rows x cols real per image, image b uses H + b*h_stride
 *         (h_stride = 0 shares one filter), natural (unshifted) DFT order
 *   out : batch x rows x cols real
 * The output does not depend on conv (each forward/inverse pair is exact).
 * ------------------------------------------------------------------------- */
int orc_pipeline(const double *img, const double *H, double *out, int64_t rows, int64_t cols,
                 int64_t batch, int64_t h_stride, int conv) {
    if (!img || !H || !out || batch < 0 || h_stride < 0) return -1;
    if (rows < 2 || cols < 2 || !is_pow2(rows) || !is_pow2(cols)) return -1;
    int64_t np = rows * cols;
    double *a = (double *)malloc(sizeof(double) * 2 * (size_t)np);
    double *s = (double *)malloc(sizeof(double) * 2 * (size_t)np);
    if (!a || !s) {
        free(a);
        free(s);
        return -2;
    }
    int rc = 0;
    for (int64_t b = 0; b < batch && !rc; ++b) {
        const double *ib = img + b * np;
        const double *hb = H + b * h_stride;
        for (int64_t i = 0; i < np; ++i) {
            a[2 * i] = ib[i];
            a[2 * i + 1] = 0.0;
        }
        rc = orc_fft2(a, s, rows, cols, 1, conv);
        if (rc) break;
        for (int64_t i = 0; i < np; ++i) {
            s[2 * i] *= hb[i];
            s[2 * i + 1] *= hb[i];
        }
        rc = orc_ifft2(s, a, rows, cols, 1, conv);
        if (rc) break;
        for (int64_t i = 0; i < np; ++i) out[b * np + i] = a[2 * i];
    }
    free(a);
    free(s);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Gradients of the Sec. 5 pipeline, y_b = Re(ifft2(H . fft2(x_b))) with the
 * per-axis convention, for an upstream gradient G_b = dL/dy_b (real).
 *
 * With W the unscaled 2D DFT matrix and s = 1/(N M), y_b = Re(A x_b) with
 * A = s W^H diag(H) W.  For real H this A is Hermitian and W is symmetric, so
 *   dL/dx_b = Re(A G_b)                      (the pipeline applied to G_b)
 *   dL/dH[k] = s sum_b Re(conj((W G_b)[k]) (W x_b)[k])
 *            = (1/s) sum_b Re(conj(F_b^G[k]) F_b^x[k])
 * where F^x = fft2(x) and F^G = fft2(G) are per-axis spectra (each = s W .).
 * H is shared by the whole batch; grad_H is summed over it.
 * ------------------------------------------------------------------------- */
int orc_pipeline_grad(const double *img, const double *H, const double *G, double *grad_img, double *grad_H,
                      int64_t rows, int64_t cols, int64_t batch) {
    if (!img || !H || !G || !grad_img || !grad_H || batch < 0) return -1;
    if (rows < 2 || cols < 2 || !is_pow2(rows) || !is_pow2(cols)) return -1;
    int64_t np = rows * cols;
    int rc = orc_pipeline(G, H, grad_img, rows, cols, batch, 0, 0);
    if (rc) return rc;
    double *a = (double *)malloc(sizeof(double) * 2 * (size_t)np);
    double *fx = (double *)malloc(sizeof(double) * 2 * (size_t)np);
    double *fg = (double *)malloc(sizeof(double) * 2 * (size_t)np);
    if (!a || !fx || !fg) {
        free(a);
        free(fx);
        free(fg);
        return -2;
    }
    double inv_s = (double)np;
    for (int64_t i = 0; i < np; ++i) grad_H[i] = 0.0;
    for (int64_t b = 0; b < batch && !rc; ++b) {
        for (int64_t i = 0; i < np; ++i) {
            a[2 * i] = img[b * np + i];
            a[2 * i + 1] = 0.0;
        }
        rc = orc_fft2(a, fx, rows, cols, 1, 0);
        if (rc) break;
        for (int64_t i = 0; i < np; ++i) {
            a[2 * i] = G[b * np + i];
            a[2 * i + 1] = 0.0;
        }
        rc = orc_fft2(a, fg, rows, cols, 1, 0);
        if (rc) break;
        for (int64_t i = 0; i < np; ++i)
            grad_H[i] += inv_s * (fg[2 * i] * fx[2 * i] + fg[2 * i + 1] * fx[2 * i + 1]);
    }
    free(a);
    free(fx);
    free(fg);
    return rc;
}
