/*
 * oracle_gemm.c -- the FP64 oracle for batched C_i += A_i * B_i.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library's product path never does, and nothing here is shared with the
 * CUDA sources (no common header, helper, table or constant).
 *
 * What it computes (paper: Alg. 1, first step C_temp = A_{V^T} * B_U, and the
 * per-entry loop nest of Alg. 2, loops 1-4, generalised to any m x n x k; the
 * low-rank factor shapes come from Eq. 1, the "(m, n, rank)" tuple of Sec. 2):
 *
 *   for every entry, for 0 <= i < m, 0 <= j < n:
 *       C[i + j*ldc] <- C[i + j*ldc] + sum_{p=0}^{k-1} A[i + p*lda] * B[p + j*ldb]
 *
 * Column-major operands with leading dimensions lda >= m, ldb >= k, ldc >= m.
 * The sum starts from the old C value and adds the k products in increasing
 * p, one rounding per multiply and one per add (compiled with
 * -ffp-contract=off so no fused multiply-add is formed).  Elements of C
 * outside the m x n window (the ld padding) are never touched.  All
 * arithmetic is IEEE binary64, as in the paper's experiments (Sec. 7, all
 * tests in double precision).
 *
 * Entries are independent, so the batch loop is parallel over entries with
 * OpenMP (the paper parallelises its outermost batch loop, loop 1A of
 * Alg. 3, across cores in the same way).
 */
#include <stddef.h>
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One entry: C(m x n) += A(m x k) * B(k x n), loop order j, p, i. */
void oracle_gemm(int32_t m, int32_t n, int32_t k,
                 const double* A, int32_t lda,
                 const double* B, int32_t ldb,
                 double* C, int32_t ldc)
{
    for (int32_t j = 0; j < n; ++j) {
        double* c = C + (size_t)j * (size_t)ldc;
        for (int32_t p = 0; p < k; ++p) {
            const double* a = A + (size_t)p * (size_t)lda;
            double b = B[(size_t)p + (size_t)j * (size_t)ldb];
            for (int32_t i = 0; i < m; ++i) {
                double prod = a[i] * b;
                c[i] = c[i] + prod;
            }
        }
    }
}

/* A batch of independent entries given as parallel arrays (one element per
 * entry).  nthreads <= 0 uses the OpenMP default.  Returns the number of
 * threads the parallel region ran with. */
int oracle_gemm_batch(int64_t count,
                      const double* const* A, const double* const* B,
                      double* const* C,
                      const int32_t* m, const int32_t* n, const int32_t* k,
                      const int32_t* lda, const int32_t* ldb, const int32_t* ldc,
                      int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < count; ++e)
            oracle_gemm(m[e], n[e], k[e], A[e], lda[e], B[e], ldb[e], C[e], ldc[e]);
    }
#else
    (void)nthreads;
    for (int64_t e = 0; e < count; ++e)
        oracle_gemm(m[e], n[e], k[e], A[e], lda[e], B[e], ldb[e], C[e], ldc[e]);
#endif
    return used;
}

/* Selected output elements only, for checks at sizes where the full oracle
 * would take too long: out[q] = c0[q] + sum_p arow[q*k + p] * bcol[q*k + p],
 * summed in increasing p exactly as oracle_gemm does for element (i, j).
 * arow holds row i of A (k values) and bcol column j of B (k values) for
 * sample q; c0 holds the old C value. */
void oracle_gemm_elements(int64_t nsamples, int32_t k,
                          const double* arow, const double* bcol,
                          const double* c0, double* out)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t q = 0; q < nsamples; ++q) {
        const double* a = arow + (size_t)q * (size_t)k;
        const double* b = bcol + (size_t)q * (size_t)k;
        double c = c0[q];
        for (int32_t p = 0; p < k; ++p) {
            double prod = a[p] * b[p];
            c = c + prod;
        }
        out[q] = c;
    }
}

/* Upper bound helper for the rounding-error bound of any summation order:
 * out[i + j*m] = |C0[i + j*ldc]| + sum_p |A[i + p*lda]| * |B[p + j*ldb]|,
 * computed in binary64 (callers add their own slack for its rounding). */
void oracle_gemm_absbound(int32_t m, int32_t n, int32_t k,
                          const double* A, int32_t lda,
                          const double* B, int32_t ldb,
                          const double* C0, int32_t ldc, double* out)
{
    for (int32_t j = 0; j < n; ++j) {
        for (int32_t i = 0; i < m; ++i)
            out[(size_t)i + (size_t)j * (size_t)m] = fabs(C0[(size_t)i + (size_t)j * (size_t)ldc]);
        for (int32_t p = 0; p < k; ++p) {
            double b = fabs(B[(size_t)p + (size_t)j * (size_t)ldb]);
            for (int32_t i = 0; i < m; ++i)
                out[(size_t)i + (size_t)j * (size_t)m] += fabs(A[(size_t)i + (size_t)p * (size_t)lda]) * b;
        }
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The low-rank multiplication core of Alg. 1 (Sec. 2): for low-rank blocks
 * A = A_U A_X A_{V^T} (rank ra) and B = B_U B_X B_{V^T} (rank rb),
 *     C_temp = A_{V^T} B_U     (ra x rb, k-long inner dimension)
 *     E_temp = A_X C_temp      (ra x rb)
 *     G_XY   = E_temp B_X      (ra x rb), written (not accumulated),
 * each step the plain product above (oracle_gemm into a zeroed target).
 * `work` holds 2 ra rb doubles. */
void oracle_lr_chain(int32_t ra, int32_t rb, int32_t k,
                     const double* AVT, int32_t ld_avt,
                     const double* BU, int32_t ld_bu,
                     const double* AX, int32_t ld_ax,
                     const double* BX, int32_t ld_bx,
                     double* G, int32_t ldg, double* work)
{
    double* Ct = work;
    double* Et = work + (size_t)ra * (size_t)rb;
    for (size_t i = 0; i < 2 * (size_t)ra * (size_t)rb; ++i) work[i] = 0.0;
    oracle_gemm(ra, rb, k, AVT, ld_avt, BU, ld_bu, Ct, ra);
    oracle_gemm(ra, rb, ra, AX, ld_ax, Ct, ra, Et, ra);
    for (int32_t j = 0; j < rb; ++j)
        for (int32_t i = 0; i < ra; ++i) G[(size_t)i + (size_t)j * (size_t)ldg] = 0.0;
    oracle_gemm(ra, rb, rb, Et, ra, BX, ld_bx, G, ldg);
}

/* A batch of chains: pointer arrays AVT, BU, AX, BX, G and per-entry
 * (ra, rb, k) with tight leading dimensions (ra, k, ra, rb, ra).
 * Parallel over entries; returns the thread count used. */
int oracle_lr_chain_batch(int64_t count,
                          const double* const* AVT, const double* const* BU,
                          const double* const* AX, const double* const* BX,
                          double* const* G,
                          const int32_t* ra, const int32_t* rb, const int32_t* k,
                          int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
        double* work = 0;
        size_t cap = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t e = 0; e < count; ++e) {
            size_t need = 2 * (size_t)ra[e] * (size_t)rb[e];
            if (need > cap) {
                free(work);
                work = (double*)malloc(need * sizeof(double));
                cap = need;
            }
            oracle_lr_chain(ra[e], rb[e], k[e], AVT[e], ra[e], BU[e], k[e], AX[e], ra[e], BX[e], rb[e],
                            G[e], ra[e], work);
        }
        free(work);
    }
#else
    (void)nthreads;
    double* work = 0;
    size_t cap = 0;
    for (int64_t e = 0; e < count; ++e) {
        size_t need = 2 * (size_t)ra[e] * (size_t)rb[e];
        if (need > cap) {
            free(work);
            work = (double*)malloc(need * sizeof(double));
            cap = need;
        }
        oracle_lr_chain(ra[e], rb[e], k[e], AVT[e], ra[e], BU[e], k[e], AX[e], ra[e], BX[e], rb[e], G[e], ra[e],
                        work);
    }
    free(work);
#endif
    return used;
}
