/*
 * Radix-2 discrete Fourier transform of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/fft.py, which the oracle's
 * linear step (App. A, Eqs. (A.3)-(A.5): transform, multiply in K-space,
 * transform back) calls.  It shares no code with the CUDA path.
 *
 * The transform is the textbook iterative Cooley-Tukey algorithm: a
 * bit-reversal permutation, then log2(n) stages that merge pairs of
 * transforms of length len/2 into one of length len,
 *     X[k]         = E[k] + w^k O[k]
 *     X[k + len/2] = E[k] - w^k O[k],     w = exp(sign 2 pi i / len),
 * with every twiddle computed directly by cos/sin in double precision (no
 * recurrence).  sign = -1 gives X_k = sum_m x_m exp(-2 pi i k m / n) (the
 * forward DFT); sign = +1 the same sum with exp(+...) and no 1/n factor.
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double kPi = 3.14159265358979323846;

/* In place on `count` contiguous rows of n complex values (re, im pairs);
 * n a power of two.  Returns 0, or -1 for an n that is not a power of two
 * or a failed allocation. */
int oracle_dft_rows(double *data, long count, long n, int sign)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    if (n == 1) return 0;
    /* twiddles w_n^k, k < n/2; stage `len` uses w_n^(k n / len) */
    double *tw = (double *)malloc(sizeof(double) * (size_t)n);
    if (!tw) return -1;
    for (long k = 0; k < n / 2; ++k) {
        const double a = sign * 2.0 * kPi * (double)k / (double)n;
        tw[2 * k] = cos(a);
        tw[2 * k + 1] = sin(a);
    }
#pragma omp parallel for schedule(static)
    for (long r = 0; r < count; ++r) {
        double *x = data + 2 * r * n;
        /* bit-reversal permutation */
        for (long i = 1, j = 0; i < n; ++i) {
            long bit = n >> 1;
            for (; j & bit; bit >>= 1) j ^= bit;
            j ^= bit;
            if (i < j) {
                const double tr = x[2 * i], ti = x[2 * i + 1];
                x[2 * i] = x[2 * j];
                x[2 * i + 1] = x[2 * j + 1];
                x[2 * j] = tr;
                x[2 * j + 1] = ti;
            }
        }
        /* butterflies */
        for (long len = 2; len <= n; len <<= 1) {
            const long half = len / 2, step = n / len;
            for (long start = 0; start < n; start += len) {
                for (long k = 0; k < half; ++k) {
                    const double wr = tw[2 * k * step], wi = tw[2 * k * step + 1];
                    double *e = x + 2 * (start + k);
                    double *o = x + 2 * (start + k + half);
                    const double br = o[0] * wr - o[1] * wi;
                    const double bi = o[0] * wi + o[1] * wr;
                    o[0] = e[0] - br;
                    o[1] = e[1] - bi;
                    e[0] = e[0] + br;
                    e[1] = e[1] + bi;
                }
            }
        }
    }
    free(tw);
    return 0;
}

/* Threads of the row loop (no effect without OpenMP); returns the count used. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
