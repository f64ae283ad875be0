/*
 * CPU oracle for the GPU compute-actor payloads -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, single-threaded C.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library; the product path
 * never does.  It shares no code, header or table with the CUDA sources.
 *
 * What it computes:
 *
 *  - Factorization (the numeric side load of the paper's mixed benchmark,
 *    Sec. 5 "Mixed Operations Under Work Load"): the plain definition of
 *    trial division.  For n >= 0 the reply is (d, n/d) for the smallest
 *    integer d >= 2 with d*d <= n and d | n; the candidates are 2 and then
 *    every odd number 3, 5, 7, ... in increasing order.  When no such d
 *    exists (n prime, or n < 4) the reply is (1, n) with status 1.
 *
 *  - Dense matrix product (the OpenCL actor of Sec. 3.6, which multiplies
 *    two square float matrices stored row-major in 1-D arrays): the exact
 *    product in float64 of the float32 inputs.  Each product of two float32
 *    values is exact in float64 (24 + 24 <= 53 significand bits); the sum
 *    over k runs in increasing k.
 *
 *  - The relative Frobenius error ||C - C64||_F / ||C64||_F in float64.
 *
 *  - A trial-division primality test, used to check factor certificates.
 *
 *  - Mandelbrot escape counts (the OpenCL actor experiment of Sec. 5,
 *    "Integrating OpenCL Actors": an image of 1920 x 1080 pixels over a cut
 *    of the complex plane, 120 or 1200 maximum iterations).  The iteration
 *    z <- z^2 + c from z = 0 in float32, each operation rounded to nearest
 *    (the library must be built with -ffp-contract=off so that no multiply
 *    and add are fused).  The count is the number of completed iterations
 *    before |z|^2 > 4 is first seen, at most max_iter.  The paper fixes
 *    neither the precision nor the order of the operations; this order
 *    (squares, escape test, cross term doubled, then the new z) is the one
 *    the GPU path follows.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

typedef unsigned __int128 u128;

/* Smallest divisor d >= 2 with d*d <= n; status 0 if found, 1 if none. */
int32_t oracle_factor(uint64_t n, uint64_t *p, uint64_t *q)
{
    if ((u128)2 * 2 <= n && n % 2 == 0) {
        *p = 2;
        *q = n / 2;
        return 0;
    }
    for (uint64_t d = 3; (u128)d * d <= n; d += 2) {
        if (n % d == 0) {
            *p = d;
            *q = n / d;
            return 0;
        }
    }
    *p = 1;
    *q = n;
    return 1;
}

void oracle_factor_batch(const uint64_t *n, int64_t count, uint64_t *p, uint64_t *q,
                         int32_t *status)
{
    for (int64_t i = 0; i < count; ++i)
        status[i] = oracle_factor(n[i], &p[i], &q[i]);
}

/* 1 if x is prime (trial division by every d with d*d <= x), else 0. */
int32_t oracle_is_prime(uint64_t x)
{
    uint64_t p, q;
    if (x < 2)
        return 0;
    return oracle_factor(x, &p, &q) == 1;
}

/* Certificate for a factor reply: p*q == n (128-bit), p <= q, and, when
 * status is 0, p and q are both prime.  Returns 1 if the certificate holds. */
int32_t oracle_check_certificate(uint64_t n, uint64_t p, uint64_t q, int32_t status)
{
    if ((u128)p * q != (u128)n)
        return 0;
    if (p > q)
        return 0;
    if (status == 1)
        return p == 1;
    return oracle_is_prime(p) && oracle_is_prime(q);
}

/* C64 = A * B, all n x n row-major; A and B float32, C64 float64. */
void oracle_gemm_f64(const float *A, const float *B, int64_t n, double *C64)
{
    for (int64_t i = 0; i < n; ++i) {
        double *row = C64 + i * n;
        for (int64_t j = 0; j < n; ++j)
            row[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double a = (double)A[i * n + k];
            const float *brow = B + k * n;
            for (int64_t j = 0; j < n; ++j)
                row[j] += a * (double)brow[j];
        }
    }
}

/* Selected rows of the product above: out[r*n + j] = C64[rows[r]][j] for
 * r < nrows, each row summed over k in increasing order as oracle_gemm_f64
 * does.  Rows of a matrix product depend only on their own row of A, so a
 * sample of rows of an n = 2048 product costs n^2 per row instead of n^3. */
void oracle_gemm_rows(const float *A, const float *B, int64_t n, const int64_t *rows, int64_t nrows,
                      double *out)
{
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double *row = out + r * n;
        for (int64_t j = 0; j < n; ++j)
            row[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double a = (double)A[i * n + k];
            const float *brow = B + k * n;
            for (int64_t j = 0; j < n; ++j)
                row[j] += a * (double)brow[j];
        }
    }
}

/* One entry C64[i][j] of the product above, same summation order. */
double oracle_gemm_entry(const float *A, const float *B, int64_t n, int64_t i, int64_t j)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k)
        s += (double)A[i * n + k] * (double)B[k * n + j];
    return s;
}

/* ||C - C64||_F / ||C64||_F over `count` entries; ||C||_F when C64 is zero. */
double oracle_rel_frobenius(const float *C, const double *C64, int64_t count)
{
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        double d = (double)C[i] - C64[i];
        num += d * d;
        den += C64[i] * C64[i];
    }
    if (den == 0.0)
        return sqrt(num);
    return sqrt(num) / sqrt(den);
}

/* Escape count of c = cx + i*cy: iterate z <- z^2 + c from z = 0, testing
 * |z|^2 = zr*zr + zi*zi > 4 before each update, for at most max_iter updates.
 * Every operation is one float32 operation rounded to nearest:
 *   x2 = zr*zr; y2 = zi*zi; stop if x2 + y2 > 4;
 *   xy = zr*zi; zi = (xy + xy) + cy; zr = (x2 - y2) + cx. */
uint32_t oracle_mandel_point(float cx, float cy, uint32_t max_iter)
{
    float zr = 0.0f, zi = 0.0f;
    uint32_t k = 0;
    while (k < max_iter) {
        float x2 = zr * zr;
        float y2 = zi * zi;
        if (x2 + y2 > 4.0f)
            break;
        float xy = zr * zi;
        zi = (xy + xy) + cy;
        zr = (x2 - y2) + cx;
        ++k;
    }
    return k;
}

/* Rows row0 .. row0+rows-1 of an image `width` pixels wide: pixel (i, j) is
 * c = (x0 + i*dx) + (y0 + j*dy) i, each coordinate one rounded product and
 * one rounded sum in float32.  out[(j - row0) * width + i] = its escape
 * count; the return value is the sum of the counts. */
uint64_t oracle_mandel_rows(float x0, float y0, float dx, float dy, uint32_t width, uint32_t row0,
                            uint32_t rows, uint32_t max_iter, uint32_t *out)
{
    uint64_t sum = 0;
    for (uint32_t r = 0; r < rows; ++r) {
        float cy = y0 + (float)(row0 + r) * dy;
        for (uint32_t i = 0; i < width; ++i) {
            float cx = x0 + (float)i * dx;
            uint32_t k = oracle_mandel_point(cx, cy, max_iter);
            out[(size_t)r * width + i] = k;
            sum += k;
        }
    }
    return sum;
}
