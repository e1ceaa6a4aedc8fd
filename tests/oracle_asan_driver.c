/*
 * Memory- and UB-safety driver for the oracle's C routines (oracle/oracle.c),
 * built with AddressSanitizer and UndefinedBehaviorSanitizer by
 * tests/test_oracle_sanitizers.py.  Test infrastructure only.
 *
 * It drives every exported routine over the shapes the tests use and their
 * edges: periodic and open cells, an empty pattern (r = 0), a dense one
 * (r above the cell diagonal), mixed block sizes 1/4/13, every op(A)/op(B)
 * combination, full and upper-only outputs, and a partial row range.  Each
 * truncated product is also checked against a dense product of the same
 * blocks restricted to the output pattern, written here independently.
 * Exit status 0 and "ok" on success.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zdouble;

int64_t or_pattern_count(int n, const double *pos, const double *cell, double r, int32_t *rowptr);
void or_pattern_fill(int n, const double *pos, const double *cell, double r, const int32_t *rowptr, int32_t *col);
void or_min_image_d2(int m, const double *pi, const double *pj, const double *cell, double *out);
void or_spgemm(int n, const int32_t *bsize,
               const int32_t *a_rp, const int32_t *a_col, const int64_t *a_off, const zdouble *a_val, int a_dag,
               const int32_t *b_rp, const int32_t *b_col, const int64_t *b_off, const zdouble *b_val, int b_dag,
               const int32_t *c_rp, const int32_t *c_col, const int64_t *c_off, zdouble *c_val,
               int row_begin, int row_end, int upper_only);

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static double urand(void) /* xorshift64*, uniform in [0, 1) */
{
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (double)((rng_state * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
}

#define CHECK(cond, ...)                                  \
    do {                                                  \
        if (!(cond)) {                                    \
            fprintf(stderr, "check failed: " __VA_ARGS__); \
            fprintf(stderr, "\n");                        \
            exit(1);                                      \
        }                                                 \
    } while (0)

typedef struct {
    int n;
    int32_t *rp, *col;
    int64_t nnzb;
} pat_t;

static pat_t make_pattern(int n, const double *pos, const double *cell, double r)
{
    pat_t p;
    p.n = n;
    p.rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    p.nnzb = or_pattern_count(n, pos, cell, r, p.rp);
    p.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p.nnzb > 0 ? p.nnzb : 1));
    or_pattern_fill(n, pos, cell, r, p.rp, p.col);
    CHECK(p.rp[0] == 0 && p.rp[n] == p.nnzb, "rowptr ends");
    for (int i = 0; i < n; ++i) {
        CHECK(p.rp[i + 1] >= p.rp[i], "rowptr monotone");
        for (int32_t q = p.rp[i] + 1; q < p.rp[i + 1]; ++q) CHECK(p.col[q] > p.col[q - 1], "columns ascending");
    }
    /* symmetric: (i,j) present iff (j,i) present */
    for (int i = 0; i < n; ++i)
        for (int32_t q = p.rp[i]; q < p.rp[i + 1]; ++q) {
            int j = p.col[q], found = 0;
            for (int32_t t = p.rp[j]; t < p.rp[j + 1]; ++t) found |= p.col[t] == i;
            CHECK(found, "pattern symmetric (%d,%d)", i, j);
        }
    return p;
}

static void free_pattern(pat_t *p)
{
    free(p->rp);
    free(p->col);
}

static int64_t *offsets(const pat_t *p, const int32_t *bs)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p->nnzb + 1));
    off[0] = 0;
    for (int i = 0; i < p->n; ++i)
        for (int32_t q = p->rp[i]; q < p->rp[i + 1]; ++q) off[q + 1] = off[q] + (int64_t)bs[i] * bs[p->col[q]];
    return off;
}

static zdouble *random_values(int64_t m)
{
    zdouble *v = (zdouble *)malloc(sizeof(zdouble) * (size_t)(m > 0 ? m : 1));
    for (int64_t e = 0; e < m; ++e) v[e] = (urand() - 0.5) + I * (urand() - 0.5);
    return v;
}

/* dense n_f x n_f copy of a block matrix */
static zdouble *to_dense(const pat_t *p, const int32_t *bs, const int *foff, int nf, const int64_t *off,
                         const zdouble *v)
{
    zdouble *d = (zdouble *)calloc((size_t)nf * nf, sizeof(zdouble));
    for (int i = 0; i < p->n; ++i)
        for (int32_t q = p->rp[i]; q < p->rp[i + 1]; ++q) {
            int j = p->col[q];
            for (int a = 0; a < bs[i]; ++a)
                for (int b = 0; b < bs[j]; ++b) d[(size_t)(foff[i] + a) * nf + foff[j] + b] = v[off[q] + a * bs[j] + b];
        }
    return d;
}

static void run_products(int n, const double *pos, const double *cell)
{
    int32_t *bs = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    static const int sizes[3] = {1, 4, 13};
    for (int i = 0; i < n; ++i) bs[i] = sizes[i % 3];
    int *foff = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    foff[0] = 0;
    for (int i = 0; i < n; ++i) foff[i + 1] = foff[i] + bs[i];
    const int nf = foff[n];

    const double radii[3][3] = {{4.0, 5.0, 6.0}, {6.0, 4.0, 5.0}, {0.0, 5.0, 100.0}};
    for (int rc = 0; rc < 3; ++rc) {
        pat_t pa = make_pattern(n, pos, cell, radii[rc][0]);
        pat_t pb = make_pattern(n, pos, cell, radii[rc][1]);
        pat_t pc = make_pattern(n, pos, cell, radii[rc][2]);
        int64_t *oa = offsets(&pa, bs), *ob = offsets(&pb, bs), *oc = offsets(&pc, bs);
        zdouble *va = random_values(oa[pa.nnzb]), *vb = random_values(ob[pb.nnzb]);
        zdouble *vc = (zdouble *)malloc(sizeof(zdouble) * (size_t)(oc[pc.nnzb] > 0 ? oc[pc.nnzb] : 1));
        zdouble *da = to_dense(&pa, bs, foff, nf, oa, va), *db = to_dense(&pb, bs, foff, nf, ob, vb);
        for (int combo = 0; combo < 4; ++combo) {
            const int adag = combo & 1, bdag = combo >> 1;
            for (int upper = 0; upper < 2; ++upper) {
                const int r0 = upper ? 1 : 0, r1 = upper ? n - 1 : n; /* a partial row range, too */
                const zdouble sentinel = 7.0 + 7.0 * I;
                for (int64_t e = 0; e < oc[pc.nnzb]; ++e) vc[e] = sentinel;
                or_spgemm(n, bs, pa.rp, pa.col, oa, va, adag, pb.rp, pb.col, ob, vb, bdag, pc.rp, pc.col, oc, vc,
                          r0, r1, upper);
                double maxref = 0.0, maxerr = 0.0;
                for (int i = 0; i < n; ++i)
                    for (int32_t q = pc.rp[i]; q < pc.rp[i + 1]; ++q) {
                        const int j = pc.col[q];
                        const int computed = i >= r0 && i < r1 && (!upper || j >= i);
                        for (int x = 0; x < bs[i]; ++x)
                            for (int y = 0; y < bs[j]; ++y) {
                                const zdouble got = vc[oc[q] + x * bs[j] + y];
                                if (!computed) {
                                    CHECK(got == sentinel, "block (%d,%d) outside the computed set was written", i, j);
                                    continue;
                                }
                                zdouble ref = 0.0;
                                const int gi = foff[i] + x, gj = foff[j] + y;
                                for (int g = 0; g < nf; ++g) {
                                    const zdouble a = adag ? conj(da[(size_t)g * nf + gi]) : da[(size_t)gi * nf + g];
                                    const zdouble b = bdag ? conj(db[(size_t)gj * nf + g]) : db[(size_t)g * nf + gj];
                                    ref += a * b;
                                }
                                maxref = fmax(maxref, cabs(ref));
                                maxerr = fmax(maxerr, cabs(got - ref));
                            }
                    }
                CHECK(maxerr <= 1e-12 * (maxref > 1.0 ? maxref : 1.0), "product mismatch %g (radii set %d, ops %d)",
                      maxerr, rc, combo);
            }
        }
        free(da);
        free(db);
        free(va);
        free(vb);
        free(vc);
        free(oa);
        free(ob);
        free(oc);
        free_pattern(&pa);
        free_pattern(&pb);
        free_pattern(&pc);
    }
    free(bs);
    free(foff);
}

int main(void)
{
    enum { N = 24 };
    double pos[3 * N];
    const double cell[3] = {9.0, 10.0, 11.0};
    for (int i = 0; i < 3 * N; ++i) pos[i] = cell[i % 3] * urand();

    /* empty pattern: no block, not even the diagonal */
    pat_t p0 = make_pattern(N, pos, cell, 0.0);
    CHECK(p0.nnzb == 0, "r = 0 gives an empty pattern");
    free_pattern(&p0);
    /* above the cell diagonal every pair is kept */
    pat_t pd = make_pattern(N, pos, cell, 100.0);
    CHECK(pd.nnzb == (int64_t)N * N, "dense pattern");
    free_pattern(&pd);

    /* minimum-image squared distances of the pairs (i, i+1): within the half cell */
    double d2[N - 1];
    or_min_image_d2(N - 1, pos, pos + 3, cell, d2);
    const double half2 = 0.25 * (cell[0] * cell[0] + cell[1] * cell[1] + cell[2] * cell[2]);
    for (int t = 0; t < N - 1; ++t) CHECK(d2[t] >= 0.0 && d2[t] <= half2 * (1.0 + 1e-12), "minimum image");

    run_products(N, pos, cell); /* periodic */
    run_products(N, pos, NULL); /* open */
    printf("ok\n");
    return 0;
}
