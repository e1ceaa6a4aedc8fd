/*
 * CPU FP64 oracle kernels for the truncated density-matrix RT-TDDFT step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code with the CUDA path.
 *
 * Two plain routines, written for obviousness rather than speed:
 *
 *  or_pattern_*  : spatial cut-off of Sec. II.A (elements between atoms
 *                  farther apart than the radius are dropped).  Block (i,j) is kept
 *                  iff the minimum-image distance of atoms i and j is strictly
 *                  below r.  Brute force over all pairs, FP64, every operation
 *                  separately rounded (compiled with -ffp-contract=off):
 *                    dx = x_j - x_i;  dx = dx - L*rint(dx/L);
 *                    d2 = (dx*dx + dy*dy) + dz*dz;  keep iff d2 < r*r.
 *
 *  or_spgemm     : truncated block product C = cut_{P_C}(op(A) * op(B)) of
 *                  the atom-blocked matrices of Sec. II.A / Sec. V.A: every
 *                  product in the method is evaluated only on the output
 *                  pattern P_C and everything outside it is dropped.
 *                    C_ij = sum_k op(A)_ik op(B)_kj   for (i,j) in P_C,
 *                  summed over k in ascending order, with op(X) = X or X^dagger
 *                  (conjugate transpose, block (k,i) of X conjugated and
 *                  transposed).  Complex FP64 throughout; real matrices are
 *                  passed with zero imaginary parts.
 *
 * Block-CSR layout: rowptr[n+1], col[nnzb] (ascending within a row),
 * voff[nnzb+1] value offsets of each row-major bi x bj block, values as
 * double complex.  Block sizes bsize[n] per atom (1, 4, 13, ... any).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zdouble;

static double min_image_d2(const double *pi, const double *pj, const double *cell)
{
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double dx = pj[d] - pi[d];
        if (cell) {
            double L = cell[d];
            dx = dx - L * rint(dx / L);
        }
        double t = dx * dx;
        d2 = (d == 0) ? t : d2 + t;
    }
    return d2;
}

/* rowptr[n+1] <- counts prefix; returns nnzb */
int64_t or_pattern_count(int n, const double *pos, const double *cell, double r, int32_t *rowptr)
{
    double r2 = r * r;
    rowptr[0] = 0;
    for (int i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int j = 0; j < n; ++j)
            if (min_image_d2(pos + 3 * i, pos + 3 * j, cell) < r2) ++c;
        rowptr[i + 1] = rowptr[i] + c;
    }
    return rowptr[n];
}

void or_pattern_fill(int n, const double *pos, const double *cell, double r,
                     const int32_t *rowptr, int32_t *col)
{
    double r2 = r * r;
    for (int i = 0; i < n; ++i) {
        int32_t q = rowptr[i];
        for (int j = 0; j < n; ++j)
            if (min_image_d2(pos + 3 * i, pos + 3 * j, cell) < r2) col[q++] = j;
    }
}

void or_min_image_d2(int m, const double *pi, const double *pj, const double *cell, double *out)
{
    for (int t = 0; t < m; ++t) out[t] = min_image_d2(pi + 3 * t, pj + 3 * t, cell);
}

/* position of column j in row i of a pattern, or -1 */
static int64_t find_block(const int32_t *rowptr, const int32_t *col, int i, int j)
{
    int32_t lo = rowptr[i], hi = rowptr[i + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    if (lo < rowptr[i + 1] && col[lo] == j) return lo;
    return -1;
}

/* element (a,b) of op(X) block (i,k): X_ik[a][b] or conj(X_ki[b][a]) */
static inline zdouble opel(const zdouble *val, const int64_t *voff, int64_t q,
                           int bcols_stored, int a, int b, int dag)
{
    if (!dag) return val[voff[q] + (int64_t)a * bcols_stored + b];
    return conj(val[voff[q] + (int64_t)b * bcols_stored + a]);
}

/*
 * C = cut_{P_C}(op(A) op(B)) for output rows [row_begin, row_end).
 * a_dag / b_dag select X^dagger.  With upper_only, only blocks with j >= i are
 * computed (others left untouched).  Rows of C are independent, so an OpenMP
 * split over rows gives results independent of the thread count.
 */
void or_spgemm(int n, const int32_t *bsize,
               const int32_t *a_rp, const int32_t *a_col, const int64_t *a_off, const zdouble *a_val, int a_dag,
               const int32_t *b_rp, const int32_t *b_col, const int64_t *b_off, const zdouble *b_val, int b_dag,
               const int32_t *c_rp, const int32_t *c_col, const int64_t *c_off, zdouble *c_val,
               int row_begin, int row_end, int upper_only)
{
#pragma omp parallel
    {
        int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        for (int j = 0; j < n; ++j) slot[j] = -1;
#pragma omp for schedule(dynamic, 1)
        for (int i = row_begin; i < row_end; ++i) {
            int bi = bsize[i];
            for (int32_t q = c_rp[i]; q < c_rp[i + 1]; ++q) {
                int j = c_col[q];
                if (upper_only && j < i) continue;
                slot[j] = q;
                int bj = bsize[j];
                for (int64_t e = 0; e < (int64_t)bi * bj; ++e) c_val[c_off[q] + e] = 0.0;
            }
            /* k runs over row i of op(A); patterns are symmetric, so column i of A
             * (for A^dagger) has the same atoms as row i. */
            for (int32_t pa = a_rp[i]; pa < a_rp[i + 1]; ++pa) {
                int k = a_col[pa];
                int bk = bsize[k];
                int64_t qa = a_dag ? find_block(a_rp, a_col, k, i) : pa;
                if (qa < 0) continue;
                int a_stride = a_dag ? bi : bk; /* stored block is (k,i): bk x bi */
                /* j runs over row k of op(B) */
                for (int32_t pb = b_rp[k]; pb < b_rp[k + 1]; ++pb) {
                    int j = b_col[pb];
                    int64_t qc = slot[j];
                    if (qc < 0) continue;
                    int bj = bsize[j];
                    int64_t qb = b_dag ? find_block(b_rp, b_col, j, k) : pb;
                    if (qb < 0) continue;
                    int b_stride = b_dag ? bk : bj; /* stored block (j,k): bj x bk */
                    zdouble *c = c_val + c_off[qc];
                    for (int x = 0; x < bi; ++x)
                        for (int y = 0; y < bj; ++y) {
                            zdouble acc = c[(int64_t)x * bj + y];
                            for (int m = 0; m < bk; ++m)
                                acc += opel(a_val, a_off, qa, a_stride, x, m, a_dag) *
                                       opel(b_val, b_off, qb, b_stride, m, y, b_dag);
                            c[(int64_t)x * bj + y] = acc;
                        }
                }
            }
            for (int32_t q = c_rp[i]; q < c_rp[i + 1]; ++q) slot[c_col[q]] = -1;
        }
        free(slot);
    }
}

int or_num_threads(void)
{
    int t = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
#endif
    return t;
}
