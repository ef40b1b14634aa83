/*
 * Oracle (test infrastructure only): plain FP64 classical matrix product.
 *
 * Computes, for the selected rows i of C (all rows when `rows` is NULL),
 *
 *     C[i, j] = alpha * sum_l A[i, l] * B[l, j] + beta * C0[i, j]
 *
 * which is the GEMM problem statement C = alpha*A*B + beta*C of Section 1
 * (Eq. 1, with the 2x2 partitioned form of Eq. 2).  Every element of A, B and
 * C0 is first converted exactly to double; the sum over l runs in FP64 in
 * increasing l.  Row-major storage throughout.
 *
 * This file is used only by tests, by the smoke check and by the CPU-baseline
 * leg of the benchmark.  Nothing on the product path links or calls it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2, ORC_F16 = 3 };

/* IEEE binary16 -> double, written from the format definition:
 * 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
static double orc_half_to_double(uint16_t h) {
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int f = h & 0x3ff;
    double v;
    if (e == 0) {
        v = ldexp((double)f, -24);            /* subnormal: f * 2^-14 * 2^-10 */
    } else if (e == 31) {
        v = f ? NAN : INFINITY;
    } else {
        v = ldexp((double)(f + 1024), e - 25); /* (1 + f/1024) * 2^(e-15) */
    }
    return sign ? -v : v;
}

/* bfloat16 -> double: the 16 bits are the top half of an IEEE binary32. */
static double orc_bf16_to_double(uint16_t b) {
    uint32_t u = ((uint32_t)b) << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

static double orc_load(const void* p, int dtype, int64_t idx) {
    switch (dtype) {
    case ORC_F64: return ((const double*)p)[idx];
    case ORC_F32: return (double)((const float*)p)[idx];
    case ORC_BF16: return orc_bf16_to_double(((const uint16_t*)p)[idx]);
    case ORC_F16: return orc_half_to_double(((const uint16_t*)p)[idx]);
    default: return NAN;
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * C_out (FP64, nrows x n, leading dimension ldo) receives the selected rows.
 * C0 may be NULL (then beta is ignored, as for beta == 0).
 * Returns 0 on success, -1 on a bad argument.
 */
int oracle_gemm(int64_t m, int64_t n, int64_t k, double alpha,
                const void* A, int a_dtype, int64_t lda,
                const void* B, int b_dtype, int64_t ldb,
                double beta, const void* C0, int c_dtype, int64_t ldc,
                double* C_out, int64_t ldo,
                const int64_t* rows, int64_t nrows) {
    if (m < 0 || n < 0 || k < 0) return -1;
    if (!rows) nrows = m;
    if (nrows < 0) return -1;
    int64_t t;
#pragma omp parallel for schedule(dynamic, 1)
    for (t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        double* out = C_out + t * ldo;
        double* acc = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (i < 0 || i >= m || !acc) {
            for (int64_t j = 0; j < n; ++j) out[j] = NAN;
            free(acc);
            continue;
        }
        /* acc[j] = sum_l A[i,l] * B[l,j], l ascending */
        for (int64_t l = 0; l < k; ++l) {
            double a = orc_load(A, a_dtype, i * lda + l);
            const int64_t brow = l * ldb;
            for (int64_t j = 0; j < n; ++j) acc[j] += a * orc_load(B, b_dtype, brow + j);
        }
        for (int64_t j = 0; j < n; ++j) {
            double c0 = (C0 && beta != 0.0) ? orc_load(C0, c_dtype, i * ldc + j) : 0.0;
            out[j] = alpha * acc[j] + (C0 && beta != 0.0 ? beta * c0 : 0.0);
        }
        free(acc);
    }
    return 0;
}
