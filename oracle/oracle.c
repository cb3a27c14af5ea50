/*
 * CPU ORACLE for masked sparse matrix-matrix products -- TEST INFRASTRUCTURE.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * load this file.  It shares no code, header, table or helper with the CUDA
 * library, and it must never be reached from the library's product path.
 *
 * What it computes (Sec. 2, "Background and Notation"): C = M .* (A B) on a
 * semiring, where only the PATTERN of the mask M is used (its values and type
 * are ignored), and the complemented form C = !M .* (A B) (Sec. 1 and the
 * complement paragraphs of Sec. 5.2 and 5.5).  An entry C_ij exists iff (i, j)
 * is allowed by the mask AND at least one k has both A_ik and B_kj stored: this
 * is the SET state of the accumulator interface (Sec. 5.1, 5.2).  Entries whose
 * numeric sum is zero are kept (structural result).
 *
 * Semirings (Sec. 2 writes the arithmetic one; graph workloads use two more):
 *   ORACLE_PT_F32 = 0 : plus-times on fp32 inputs, accumulated in fp64 (each
 *                       fp32 x fp32 product is exact in fp64); also returns
 *                       S_ij = sum |a_ik| |b_kj| for error bounds.
 *   ORACLE_PT_I64 = 1 : plus-times on int64, two's-complement wrap mod 2^64.
 *   ORACLE_PP_I64 = 2 : plus-pair: every matching k contributes 1.
 *
 * Two independent algorithms:
 *   ORACLE_MERGE = 0 : pull / inner-product form (Sec. 4.1): for each allowed
 *                      (i, j) of a non-complemented mask, a sorted two-pointer
 *                      merge of row A_i* with column B_*j (B transposed by a
 *                      stable counting sort).  Non-complemented only.
 *   ORACLE_ESC   = 1 : expand-sort-compress per row: all triples (j, k, a*b)
 *                      from A_i* x B_k*, sorted by (j, k), reduced by j (same
 *                      ascending-k summation order as the merge), then kept or
 *                      dropped by a merge with the sorted mask row.  Both mask
 *                      forms.
 * Output rows are canonical CSR: columns ascending.
 *
 * Gradients of l = sum_ij G_ij C_ij for C = M .* (A B) (fp32 inputs, fp64
 * arithmetic): dA_ik = sum_j G_ij B_kj for stored (i, k) of A, and
 * dB_kj = sum_i A_ik G_ij for stored (k, j) of B, with G stored on C's pattern.
 *
 * Plain C99 + OpenMP (dynamic schedule over rows).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the parallel loops below from now on (n >= 1); the oracle's
 * results do not depend on it.  Used to time the oracle on one core. */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

enum { ORACLE_PT_F32 = 0, ORACLE_PT_I64 = 1, ORACLE_PP_I64 = 2 };
enum { ORACLE_MERGE = 0, ORACLE_ESC = 1 };
enum { ORACLE_OK = 0, ORACLE_BAD_ROWPTR = 1, ORACLE_BAD_COL = 2, ORACLE_UNSORTED = 3,
       ORACLE_BAD_ARGS = 4, ORACLE_NOMEM = 5 };

typedef struct {
    int64_t nrows;     /* rows in this result (all rows, or the selected ones) */
    int64_t *rowptr;   /* nrows + 1 */
    int32_t *colidx;
    double *vf;        /* PT_F32 values (fp64) */
    int64_t *vi;       /* PT_I64 / PP_I64 values */
    double *S;         /* PT_F32: sum |a| |b| per entry */
} oracle_result;

/* ---- step 1: validation ---------------------------------------------- */
int oracle_validate_csr(int64_t nrows, int64_t ncols, const int32_t *rp, const int32_t *ci) {
    if (nrows < 0 || ncols < 0) return ORACLE_BAD_ARGS;
    if (nrows > 0 && rp[0] != 0) return ORACLE_BAD_ROWPTR;
    for (int64_t i = 0; i < nrows; ++i) {
        if (rp[i + 1] < rp[i]) return ORACLE_BAD_ROWPTR;
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (ci[t] < 0 || ci[t] >= ncols) return ORACLE_BAD_COL;
            if (t > rp[i] && ci[t] <= ci[t - 1]) return ORACLE_UNSORTED;
        }
    }
    return ORACLE_OK;
}

/* ---- step 2: stable counting-sort transpose (rows ascending per column) -- */
static int transpose(int64_t nrows, int64_t ncols, const int32_t *rp, const int32_t *ci,
                     int64_t **trp_out, int32_t **tci_out, int64_t **tsrc_out) {
    int64_t nnz = nrows > 0 ? rp[nrows] : 0;
    int64_t *trp = (int64_t *)calloc((size_t)ncols + 1, sizeof(int64_t));
    int32_t *tci = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int64_t *tsrc = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc(((size_t)ncols + 1) * sizeof(int64_t));
    if (!trp || !tci || !tsrc || !pos) { free(trp); free(tci); free(tsrc); free(pos); return ORACLE_NOMEM; }
    for (int64_t t = 0; t < nnz; ++t) trp[ci[t] + 1]++;
    for (int64_t j = 0; j < ncols; ++j) trp[j + 1] += trp[j];
    memcpy(pos, trp, ((size_t)ncols + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nrows; ++i)
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
            int64_t w = pos[ci[t]]++;
            tci[w] = (int32_t)i;   /* row index of the entry */
            tsrc[w] = t;           /* position of the entry in the CSR arrays */
        }
    free(pos);
    *trp_out = trp; *tci_out = tci; *tsrc_out = tsrc;
    return ORACLE_OK;
}

static int binsearch(const int32_t *a, int64_t len, int32_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == x;
}

/* Per-row temporary result. */
typedef struct { int64_t len; int32_t *col; double *vf; int64_t *vi; double *S; } row_out;

static void row_alloc(row_out *r, int64_t cap, int sr) {
    size_t c = (size_t)(cap > 0 ? cap : 1);
    r->len = 0;
    r->col = (int32_t *)malloc(c * sizeof(int32_t));
    r->vf = (sr == ORACLE_PT_F32) ? (double *)malloc(c * sizeof(double)) : NULL;
    r->S = (sr == ORACLE_PT_F32) ? (double *)malloc(c * sizeof(double)) : NULL;
    r->vi = (sr != ORACLE_PT_F32) ? (int64_t *)malloc(c * sizeof(int64_t)) : NULL;
}

/* ---- step 3: non-complemented, sorted merge per allowed (i, j) ---------- */
static void row_merge(int sr, int64_t i, const int32_t *Mrp, const int32_t *Mci,
                      const int32_t *Arp, const int32_t *Aci, const void *Av,
                      const int64_t *Btrp, const int32_t *Btci, const int64_t *Btsrc, const void *Bv,
                      row_out *out) {
    int64_t mlen = Mrp[i + 1] - Mrp[i];
    row_alloc(out, mlen, sr);
    for (int64_t q = Mrp[i]; q < Mrp[i + 1]; ++q) {
        int32_t j = Mci[q];
        int64_t pa = Arp[i], ea = Arp[i + 1];
        int64_t pb = Btrp[j], eb = Btrp[j + 1];
        int64_t matches = 0;
        double sf = 0.0, sabs = 0.0;
        uint64_t si = 0;
        while (pa < ea && pb < eb) {
            int32_t ka = Aci[pa], kb = Btci[pb];
            if (ka < kb) { ++pa; continue; }
            if (kb < ka) { ++pb; continue; }
            /* A_ik and B_kj both stored: one product */
            ++matches;
            if (sr == ORACLE_PT_F32) {
                double a = (double)((const float *)Av)[pa];
                double b = (double)((const float *)Bv)[Btsrc[pb]];
                sf += a * b;
                sabs += fabs(a) * fabs(b);
            } else if (sr == ORACLE_PT_I64) {
                uint64_t a = (uint64_t)((const int64_t *)Av)[pa];
                uint64_t b = (uint64_t)((const int64_t *)Bv)[Btsrc[pb]];
                si += a * b;
            } else {
                si += 1;
            }
            ++pa; ++pb;
        }
        if (matches > 0) {
            int64_t w = out->len++;
            out->col[w] = j;
            if (sr == ORACLE_PT_F32) { out->vf[w] = sf; out->S[w] = sabs; }
            else out->vi[w] = (int64_t)si;
        }
    }
}

/* ---- step 4: expand-sort-compress per row, then mask filter -------------- */
typedef struct { int32_t j, k; double vf, S; uint64_t vi; } triple;

static int cmp_triple(const void *x, const void *y) {
    const triple *a = (const triple *)x, *b = (const triple *)y;
    if (a->j != b->j) return (a->j > b->j) - (a->j < b->j);
    return (a->k > b->k) - (a->k < b->k);
}

static int row_esc(int sr, int complement, int64_t i, const int32_t *Mrp, const int32_t *Mci,
                   const int32_t *Arp, const int32_t *Aci, const void *Av,
                   const int32_t *Brp, const int32_t *Bci, const void *Bv, row_out *out) {
    int64_t nt = 0;
    for (int64_t pa = Arp[i]; pa < Arp[i + 1]; ++pa) nt += Brp[Aci[pa] + 1] - Brp[Aci[pa]];
    triple *T = (triple *)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(triple));
    if (!T) return ORACLE_NOMEM;
    int64_t w = 0;
    for (int64_t pa = Arp[i]; pa < Arp[i + 1]; ++pa) {
        int32_t k = Aci[pa];
        for (int64_t pb = Brp[k]; pb < Brp[k + 1]; ++pb) {
            triple *t = &T[w++];
            t->j = Bci[pb]; t->k = k; t->vf = 0.0; t->S = 0.0; t->vi = 0;
            if (sr == ORACLE_PT_F32) {
                double a = (double)((const float *)Av)[pa], b = (double)((const float *)Bv)[pb];
                t->vf = a * b; t->S = fabs(a) * fabs(b);
            } else if (sr == ORACLE_PT_I64) {
                t->vi = (uint64_t)((const int64_t *)Av)[pa] * (uint64_t)((const int64_t *)Bv)[pb];
            } else {
                t->vi = 1;
            }
        }
    }
    if (nt > 1) qsort(T, (size_t)nt, sizeof(triple), cmp_triple);
    row_alloc(out, nt, sr);
    const int32_t *mrow = Mci + Mrp[i];
    int64_t mlen = Mrp[i + 1] - Mrp[i];
    for (int64_t s = 0; s < nt;) {
        int64_t e = s;
        double vf = 0.0, S = 0.0;
        uint64_t vi = 0;
        while (e < nt && T[e].j == T[s].j) { vf += T[e].vf; S += T[e].S; vi += T[e].vi; ++e; }
        int in_mask = binsearch(mrow, mlen, T[s].j);
        if (in_mask != complement) {
            int64_t o = out->len++;
            out->col[o] = T[s].j;
            if (sr == ORACLE_PT_F32) { out->vf[o] = vf; out->S[o] = S; }
            else out->vi[o] = (int64_t)vi;
        }
        s = e;
    }
    free(T);
    return ORACLE_OK;
}

static void result_free_rows(row_out *rows, int64_t n) {
    for (int64_t r = 0; r < n; ++r) { free(rows[r].col); free(rows[r].vf); free(rows[r].vi); free(rows[r].S); }
    free(rows);
}

/* Computes C (or the selected rows of C; rows_sel may be NULL).  Returns
 * NULL and sets *err on invalid arguments.  Mask values are never read. */
oracle_result *oracle_masked_spgemm(int sr, int complement, int method,
                                    int64_t m, int64_t k, int64_t n,
                                    const int32_t *Mrp, const int32_t *Mci,
                                    const int32_t *Arp, const int32_t *Aci, const void *Av,
                                    const int32_t *Brp, const int32_t *Bci, const void *Bv,
                                    int64_t nsel, const int32_t *rows_sel, int *err) {
    *err = ORACLE_OK;
    if (sr < 0 || sr > 2 || (method == ORACLE_MERGE && complement) || m < 0 || k < 0 || n < 0) {
        *err = ORACLE_BAD_ARGS; return NULL;
    }
    if ((*err = oracle_validate_csr(m, n, Mrp, Mci)) || (*err = oracle_validate_csr(m, k, Arp, Aci)) ||
        (*err = oracle_validate_csr(k, n, Brp, Bci)))
        return NULL;
    int64_t nr = rows_sel ? nsel : m;
    if (rows_sel)
        for (int64_t r = 0; r < nr; ++r)
            if (rows_sel[r] < 0 || rows_sel[r] >= m) { *err = ORACLE_BAD_ARGS; return NULL; }
    int64_t *Btrp = NULL, *Btsrc = NULL;
    int32_t *Btci = NULL;
    if (method == ORACLE_MERGE && (*err = transpose(k, n, Brp, Bci, &Btrp, &Btci, &Btsrc))) return NULL;

    row_out *rows = (row_out *)calloc((size_t)(nr > 0 ? nr : 1), sizeof(row_out));
    int fail = 0;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows_sel ? rows_sel[r] : r;
        if (method == ORACLE_MERGE)
            row_merge(sr, i, Mrp, Mci, Arp, Aci, Av, Btrp, Btci, Btsrc, Bv, &rows[r]);
        else if (row_esc(sr, complement, i, Mrp, Mci, Arp, Aci, Av, Brp, Bci, Bv, &rows[r]))
            fail = 1;
    }
    free(Btrp); free(Btci); free(Btsrc);
    if (fail) { result_free_rows(rows, nr); *err = ORACLE_NOMEM; return NULL; }

    /* step 5: canonical CSR */
    oracle_result *res = (oracle_result *)calloc(1, sizeof(oracle_result));
    res->nrows = nr;
    res->rowptr = (int64_t *)malloc(((size_t)nr + 1) * sizeof(int64_t));
    res->rowptr[0] = 0;
    for (int64_t r = 0; r < nr; ++r) res->rowptr[r + 1] = res->rowptr[r] + rows[r].len;
    int64_t nnz = res->rowptr[nr];
    size_t c = (size_t)(nnz > 0 ? nnz : 1);
    res->colidx = (int32_t *)malloc(c * sizeof(int32_t));
    if (sr == ORACLE_PT_F32) { res->vf = (double *)malloc(c * sizeof(double)); res->S = (double *)malloc(c * sizeof(double)); }
    else res->vi = (int64_t *)malloc(c * sizeof(int64_t));
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t o = res->rowptr[r], len = rows[r].len;
        memcpy(res->colidx + o, rows[r].col, (size_t)len * sizeof(int32_t));
        if (sr == ORACLE_PT_F32) {
            memcpy(res->vf + o, rows[r].vf, (size_t)len * sizeof(double));
            memcpy(res->S + o, rows[r].S, (size_t)len * sizeof(double));
        } else {
            memcpy(res->vi + o, rows[r].vi, (size_t)len * sizeof(int64_t));
        }
    }
    result_free_rows(rows, nr);
    return res;
}

int64_t oracle_result_nrows(const oracle_result *r) { return r->nrows; }
int64_t oracle_result_nnz(const oracle_result *r) { return r->rowptr[r->nrows]; }

/* Copies the result out; any destination pointer may be NULL. */
void oracle_result_copy(const oracle_result *r, int64_t *rowptr, int32_t *colidx, void *values, double *S) {
    int64_t nnz = r->rowptr[r->nrows];
    if (rowptr) memcpy(rowptr, r->rowptr, ((size_t)r->nrows + 1) * sizeof(int64_t));
    if (colidx) memcpy(colidx, r->colidx, (size_t)nnz * sizeof(int32_t));
    if (values) {
        if (r->vf) memcpy(values, r->vf, (size_t)nnz * sizeof(double));
        else memcpy(values, r->vi, (size_t)nnz * sizeof(int64_t));
    }
    if (S && r->S) memcpy(S, r->S, (size_t)nnz * sizeof(double));
}

void oracle_result_free(oracle_result *r) {
    if (!r) return;
    free(r->rowptr); free(r->colidx); free(r->vf); free(r->vi); free(r->S); free(r);
}

/* ---- step 7: gradients of l = sum G_ij C_ij (fp32 inputs, fp64 sums) ----- */
/* A: m x k, B: k x n, G: m x n (stored on C's pattern).  dA has nnz(A)
 * entries aligned with A's storage, dB has nnz(B) entries aligned with B's. */
int oracle_grad(int64_t m, int64_t k, int64_t n,
                const int32_t *Arp, const int32_t *Aci, const float *Av,
                const int32_t *Brp, const int32_t *Bci, const float *Bv,
                const int32_t *Grp, const int32_t *Gci, const float *Gv,
                double *dA, double *dB) {
    int err;
    if ((err = oracle_validate_csr(m, k, Arp, Aci)) || (err = oracle_validate_csr(k, n, Brp, Bci)) ||
        (err = oracle_validate_csr(m, n, Grp, Gci)))
        return err;
    /* dA_ik = <G_i*, B_k*>: merge of two sorted rows */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t t = Arp[i]; t < Arp[i + 1]; ++t) {
            int32_t kk = Aci[t];
            int64_t pg = Grp[i], eg = Grp[i + 1], pb = Brp[kk], eb = Brp[kk + 1];
            double s = 0.0;
            while (pg < eg && pb < eb) {
                if (Gci[pg] < Bci[pb]) ++pg;
                else if (Bci[pb] < Gci[pg]) ++pb;
                else { s += (double)Gv[pg] * (double)Bv[pb]; ++pg; ++pb; }
            }
            dA[t] = s;
        }
    }
    /* dB_kj = <A_*k, G_*j>: merge of column k of A with column j of G */
    int64_t *Atrp, *Atsrc, *Gtrp, *Gtsrc;
    int32_t *Atci, *Gtci;
    if ((err = transpose(m, k, Arp, Aci, &Atrp, &Atci, &Atsrc))) return err;
    if ((err = transpose(m, n, Grp, Gci, &Gtrp, &Gtci, &Gtsrc))) {
        free(Atrp); free(Atci); free(Atsrc); return err;
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t kk = 0; kk < k; ++kk) {
        for (int64_t t = Brp[kk]; t < Brp[kk + 1]; ++t) {
            int32_t j = Bci[t];
            int64_t pa = Atrp[kk], ea = Atrp[kk + 1], pg = Gtrp[j], eg = Gtrp[j + 1];
            double s = 0.0;
            while (pa < ea && pg < eg) {
                if (Atci[pa] < Gtci[pg]) ++pa;
                else if (Gtci[pg] < Atci[pa]) ++pg;
                else { s += (double)Av[Atsrc[pa]] * (double)Gv[Gtsrc[pg]]; ++pa; ++pg; }
            }
            dB[t] = s;
        }
    }
    free(Atrp); free(Atci); free(Atsrc); free(Gtrp); free(Gtci); free(Gtsrc);
    return ORACLE_OK;
}

/* ---- betweenness centrality (Brandes), the application of Sec. 8.3 ------
 * For each source s of the batch: a breadth-first search from s gives each
 * reached vertex v its level and sigma_sv, the number of shortest s-v paths
 * (sigma_s = 1; sigma_w = sum of sigma_v over v -> w edges with
 * level(v) = level(w) - 1); then, in decreasing level order, the dependency
 * delta_s(v) = sum over v -> w edges with level(w) = level(v) + 1 of
 * sigma_v / sigma_w * (1 + delta_s(w)).  bc(v) = sum over the sources s != v
 * of delta_s(v).  Edges are the stored entries of the n x n CSR (v -> w for
 * entry (v, w)); values are ignored.  fp64 throughout; sources in parallel. */
int oracle_bc(int64_t n, const int32_t *rp, const int32_t *ci, int64_t nsrc, const int32_t *src, double *bc) {
    int err;
    if ((err = oracle_validate_csr(n, n, rp, ci))) return err;
    for (int64_t s = 0; s < nsrc; ++s)
        if (src[s] < 0 || src[s] >= n) return ORACLE_BAD_ARGS;
    for (int64_t v = 0; v < n; ++v) bc[v] = 0.0;
    int failed = 0;
    #pragma omp parallel
    {
        int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        double *sigma = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double *delta = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double *local = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!level || !order || !sigma || !delta || !local) {
            #pragma omp atomic write
            failed = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t s = 0; s < nsrc; ++s) {
                for (int64_t v = 0; v < n; ++v) { level[v] = -1; sigma[v] = 0.0; delta[v] = 0.0; }
                int64_t head = 0, tail = 0;
                const int32_t s0 = src[s];
                level[s0] = 0;
                sigma[s0] = 1.0;
                order[tail++] = s0;
                while (head < tail) {                 /* BFS; order = visit order */
                    const int32_t v = order[head++];
                    for (int64_t t = rp[v]; t < rp[v + 1]; ++t) {
                        const int32_t w = ci[t];
                        if (level[w] < 0) { level[w] = level[v] + 1; order[tail++] = w; }
                        if (level[w] == level[v] + 1) sigma[w] += sigma[v];
                    }
                }
                for (int64_t x = tail - 1; x >= 0; --x) {   /* decreasing level */
                    const int32_t v = order[x];
                    double d = 0.0;
                    for (int64_t t = rp[v]; t < rp[v + 1]; ++t) {
                        const int32_t w = ci[t];
                        if (level[w] == level[v] + 1) d += sigma[v] / sigma[w] * (1.0 + delta[w]);
                    }
                    delta[v] = d;
                    if (v != s0) local[v] += d;
                }
            }
            #pragma omp critical
            for (int64_t v = 0; v < n; ++v) bc[v] += local[v];
        }
        free(level); free(order); free(sigma); free(delta); free(local);
    }
    return failed ? ORACLE_NOMEM : ORACLE_OK;
}

/* ---- k-truss, the application of Sec. 8.2: the largest subgraph in which
 * every edge (u, v) lies on at least k - 2 triangles of the subgraph.
 * Support of a kept edge = number of w with (u, w) and (v, w) both kept (a
 * merge of the two kept neighbour rows); edges below k - 2 are removed, and
 * the supports recomputed, until nothing changes.  A is a symmetric n x n
 * pattern; self loops are never kept.  keep[e] = 1 for the stored entries of
 * the k-truss, support[e] their final support (0 where not kept). */
int oracle_ktruss(int64_t n, const int32_t *rp, const int32_t *ci, int64_t k, uint8_t *keep, int64_t *support,
                  int64_t *iterations) {
    int err;
    if ((err = oracle_validate_csr(n, n, rp, ci))) return err;
    const int64_t nnz = rp[n];
    for (int64_t v = 0; v < n; ++v)
        for (int64_t t = rp[v]; t < rp[v + 1]; ++t) keep[t] = ci[t] != v;
    int64_t it = 0;
    for (;;) {
        ++it;
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t u = 0; u < n; ++u) {
            for (int64_t t = rp[u]; t < rp[u + 1]; ++t) {
                support[t] = 0;
                if (!keep[t]) continue;
                const int32_t v = ci[t];
                int64_t a = rp[u], ea = rp[u + 1], b = rp[v], eb = rp[v + 1], s = 0;
                while (a < ea && b < eb) {
                    if (!keep[a]) { ++a; continue; }
                    if (!keep[b]) { ++b; continue; }
                    if (ci[a] < ci[b]) ++a;
                    else if (ci[b] < ci[a]) ++b;
                    else { ++s; ++a; ++b; }
                }
                support[t] = s;
            }
        }
        int64_t removed = 0;
        for (int64_t t = 0; t < nnz; ++t)
            if (keep[t] && support[t] < k - 2) { keep[t] = 0; ++removed; }
        if (!removed) break;
    }
    for (int64_t t = 0; t < nnz; ++t)
        if (!keep[t]) support[t] = 0;
    *iterations = it;
    return ORACLE_OK;
}
