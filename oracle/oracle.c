/*
 * CPU oracle for the batched parallel-prefix operations (test infrastructure).
 *
 * This file is test infrastructure, not part of the library: only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may build, load
 * or call it.  It shares no code, header, table or helper with the CUDA path.
 * Everything here is the plain, slow definition of each operation, written so
 * that it can be checked against the paper by eye:
 *
 *   - scan:    Section III, "Scan Operator" -- each element is replaced by the
 *              accumulated sum from the first element up to itself (inclusive).
 *   - FFT:     Section III, "Fast Fourier Transform" -- the complex DFT
 *              X[k] = sum_j x[j] exp(s * 2 pi i j k / N), s = -1 forward,
 *              s = +1 inverse (unnormalised); computed by recursive radix-2
 *              decimation-in-time Cooley-Tukey, and by the O(N^2) sum.
 *   - tridiag: Section III, "Tridiagonal system solvers" --
 *              a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, solved by the Thomas
 *              algorithm (Gaussian elimination without pivoting, which is
 *              stable for strictly diagonally dominant rows).
 *
 * Layout: every batched array is row-major [batch][n].  Complex values are
 * interleaved (re, im) pairs of doubles.  a[s][0] and c[s][n-1] are outside
 * the matrix and are never read.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Inclusive int32 scan with two's-complement wrap-around (mod 2^32):
 * the accumulator is uint32_t, so overflow is defined behaviour. */
void oracle_scan_i32(const int32_t *x, int32_t *y, int64_t n, int64_t batch)
{
    for (int64_t s = 0; s < batch; ++s) {
        uint32_t acc = 0;
        for (int64_t i = 0; i < n; ++i) {
            acc += (uint32_t)x[s * n + i];
            y[s * n + i] = (int32_t)acc;
        }
    }
}

/* Inclusive float32 scan, accumulated sequentially in float64.
 * The output is the float64 running sum (the caller rounds if it wants). */
void oracle_scan_f32(const float *x, double *y, int64_t n, int64_t batch)
{
    for (int64_t s = 0; s < batch; ++s) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            acc += (double)x[s * n + i];
            y[s * n + i] = acc;
        }
    }
}

/* One recursive radix-2 decimation-in-time step on n points read from
 * in[0], in[stride], in[2*stride], ...; writes n points contiguously to out.
 * X[k]       = E[k] + w^k O[k]
 * X[k + n/2] = E[k] - w^k O[k],  w = exp(sign * 2 pi i / n). */
static void fft_rec(const double *in, int64_t stride, double *out, int64_t n,
                    int sign, double *tmp)
{
    if (n == 1) {
        out[0] = in[0];
        out[1] = in[1];
        return;
    }
    int64_t h = n / 2;
    double *even = tmp;          /* h complex */
    double *odd = tmp + 2 * h;   /* h complex */
    double *sub = tmp + 4 * h;   /* scratch for the recursion */
    fft_rec(in, 2 * stride, even, h, sign, sub);
    fft_rec(in + 2 * stride, 2 * stride, odd, h, sign, sub);
    for (int64_t k = 0; k < h; ++k) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        double wr = cos(ang), wi = sin(ang);
        double or_ = odd[2 * k], oi = odd[2 * k + 1];
        double tr = wr * or_ - wi * oi;
        double ti = wr * oi + wi * or_;
        out[2 * k] = even[2 * k] + tr;
        out[2 * k + 1] = even[2 * k + 1] + ti;
        out[2 * (k + h)] = even[2 * k] - tr;
        out[2 * (k + h) + 1] = even[2 * k + 1] - ti;
    }
}

/* Batched complex DFT of power-of-two length n by recursive radix-2 FFT.
 * dir = -1: forward (exp(-2 pi i jk/N)); dir = +1: inverse, unnormalised.
 * Returns 0, or -1 if n is not a power of two or memory runs out. */
int oracle_fft_f64(const double *x, double *X, int64_t n, int64_t batch, int dir)
{
    if (n < 1 || (n & (n - 1)) != 0 || (dir != -1 && dir != 1))
        return -1;
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)(4 * n + 8));
    if (!tmp)
        return -1;
    for (int64_t s = 0; s < batch; ++s)
        fft_rec(x + 2 * s * n, 1, X + 2 * s * n, n, dir, tmp);
    free(tmp);
    return 0;
}

/* Batched complex DFT by the O(N^2) definition, accumulated in long double
 * with the phase reduced exactly as (j*k mod N)/N.  Any length n >= 1. */
void oracle_dft_f64(const double *x, double *X, int64_t n, int64_t batch, int dir)
{
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int64_t s = 0; s < batch; ++s) {
        const double *xs = x + 2 * s * n;
        for (int64_t k = 0; k < n; ++k) {
            long double re = 0.0L, im = 0.0L;
            for (int64_t j = 0; j < n; ++j) {
                int64_t m = (j * k) % n;
                long double ang = (long double)dir * two_pi * (long double)m / (long double)n;
                long double c = cosl(ang), sn = sinl(ang);
                re += (long double)xs[2 * j] * c - (long double)xs[2 * j + 1] * sn;
                im += (long double)xs[2 * j] * sn + (long double)xs[2 * j + 1] * c;
            }
            X[2 * (s * n + k)] = (double)re;
            X[2 * (s * n + k) + 1] = (double)im;
        }
    }
}

/* Batched Thomas algorithm in float64 on float32 coefficients (widened).
 * Forward sweep: c'_i = c_i / m_i, d'_i = (d_i - a_i d'_{i-1}) / m_i with
 * m_i = b_i - a_i c'_{i-1}; back substitution x_i = d'_i - c'_i x_{i+1}.
 * a[s][0] and c[s][n-1] are never read.  Returns 0, or -1 on bad arguments. */
int oracle_thomas_f64(const float *a, const float *b, const float *c, const float *d,
                      double *x, int64_t n, int64_t batch)
{
    if (n < 1)
        return -1;
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double *dp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!cp || !dp) {
        free(cp);
        free(dp);
        return -1;
    }
    for (int64_t s = 0; s < batch; ++s) {
        const float *as = a + s * n, *bs = b + s * n, *cs = c + s * n, *ds = d + s * n;
        double *xs = x + s * n;
        for (int64_t i = 0; i < n; ++i) {
            double ai = (i > 0) ? (double)as[i] : 0.0;
            double ci = (i < n - 1) ? (double)cs[i] : 0.0;
            double cprev = (i > 0) ? cp[i - 1] : 0.0;
            double dprev = (i > 0) ? dp[i - 1] : 0.0;
            double m = (double)bs[i] - ai * cprev;
            cp[i] = ci / m;
            dp[i] = ((double)ds[i] - ai * dprev) / m;
        }
        xs[n - 1] = dp[n - 1];
        for (int64_t i = n - 2; i >= 0; --i)
            xs[i] = dp[i] - cp[i] * xs[i + 1];
    }
    free(cp);
    free(dp);
    return 0;
}
