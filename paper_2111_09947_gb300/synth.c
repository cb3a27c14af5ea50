/*
 * Seeded synthetic inputs for masked SpGEMM workloads.
 *
 * This module builds the matrices the library is exercised on: Erdos-Renyi
 * and R-MAT graphs (Sec. 7, "Experimental Setup": Graph500 R-MAT parameters),
 * CSR assembly with symmetrisation / de-duplication / self-loop removal,
 * the degree relabelling used before triangle counting (Sec. 8.2), and the
 * two-level multi-source BFS frontiers that feed a complemented-mask step of
 * betweenness centrality (Sec. 8.4).  It contains none of the masked-product
 * arithmetic: it only produces inputs, and both the CUDA path and the CPU
 * oracle consume the bytes it writes.
 *
 * Random numbers come from one counter-based generator, SplitMix64
 * (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014; the 64-bit finaliser as published by S. Vigna):
 * the i-th draw of a stream with key K is mix(K + (i + 1) * GAMMA).  Every
 * draw is addressed by (key, index), so results do not depend on thread
 * count or scheduling.
 *
 * All functions are plain C99 with OpenMP pragmas; they compile and give the
 * same results on x86-64 and AArch64 (integer paths are exact; the few libm
 * calls only shape patterns and values that are generated once per run).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define SM_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output of a SplitMix64 stream whose state starts at `key`. */
static inline uint64_t sm_draw(uint64_t key, uint64_t i) {
    return sm_mix(key + (i + 1) * SM_GAMMA);
}

/* Key of stream `stream` under base seed `seed`. */
uint64_t synth_key(uint64_t seed, uint64_t stream) {
    return sm_mix(sm_mix(seed + SM_GAMMA) ^ sm_mix(stream * 0xD1B54A32D192ED03ULL + SM_GAMMA));
}

uint64_t synth_draw(uint64_t key, uint64_t i) { return sm_draw(key, i); }

/* Uniform fp32 in [-1, 1) on a 2^-23 grid: exactly representable in fp32. */
void synth_uniform_f32(uint64_t key, int64_t count, float *out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        uint64_t r = sm_draw(key, (uint64_t)i);
        out[i] = (float)((double)(r >> 40) * (1.0 / 8388608.0) - 1.0);
    }
}

/* Standard normal fp32 by the Box-Muller transform on draws (2i, 2i+1). */
void synth_normal_f32(uint64_t key, int64_t count, float *out) {
    const double two_pi = 6.283185307179586476925286766559;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        uint64_t r1 = sm_draw(key, 2 * (uint64_t)i);
        uint64_t r2 = sm_draw(key, 2 * (uint64_t)i + 1);
        double u1 = ((double)(r1 >> 11) + 1.0) * (1.0 / 9007199254740992.0); /* (0, 1] */
        double u2 = (double)(r2 >> 11) * (1.0 / 9007199254740992.0);         /* [0, 1) */
        out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
    }
}

/* ------------------------------------------------------------------------ */
/* Erdos-Renyi G(m x n, p = d / n): every (i, j) present independently with   */
/* probability p.  Row i walks the columns with geometric gaps drawn from the */
/* row's own stream, which yields exactly a Bernoulli(p) pattern, sorted.     */

static int64_t er_row(uint64_t key, int64_t i, int64_t n, double p, int32_t *out) {
    int64_t cnt = 0;
    if (p >= 1.0) {
        for (int64_t j = 0; j < n; ++j) { if (out) out[cnt] = (int32_t)j; ++cnt; }
        return cnt;
    }
    if (p <= 0.0 || n == 0) return 0;
    uint64_t rk = sm_draw(key, (uint64_t)i);
    double lq = log1p(-p);
    int64_t j = -1;
    for (uint64_t t = 0;; ++t) {
        double u = ((double)(sm_draw(rk, t) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        double g = floor(log(u) / lq);
        if (g >= (double)n) break;
        j += 1 + (int64_t)g;
        if (j >= n) break;
        if (out) out[cnt] = (int32_t)j;
        ++cnt;
    }
    return cnt;
}

/* Pass 1: row counts into rowptr[1..m]; returns nnz.  rowptr is int64 here. */
int64_t synth_er_count(uint64_t key, int64_t m, int64_t n, double d, int64_t *rowptr) {
    double p = (n > 0) ? d / (double)n : 0.0;
    rowptr[0] = 0;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) rowptr[i + 1] = er_row(key, i, n, p, NULL);
    for (int64_t i = 0; i < m; ++i) rowptr[i + 1] += rowptr[i];
    return rowptr[m];
}

/* Pass 2: column indices for the counts of pass 1. */
void synth_er_fill(uint64_t key, int64_t m, int64_t n, double d, const int64_t *rowptr, int32_t *colidx) {
    double p = (n > 0) ? d / (double)n : 0.0;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) er_row(key, i, n, p, colidx + rowptr[i]);
}

/* ------------------------------------------------------------------------ */
/* R-MAT edge list (Chakrabarti et al.; Graph500 quadrant probabilities a, b, */
/* c, d = 1 - a - b - c).  Each edge takes `scale` quadrant choices, four per */
/* 64-bit draw (16 bits each); bit `scale-1-l` of (src, dst) is set by the    */
/* l-th choice.  Endpoints >= n are rejected (n need not be a power of two).  */
/* Returns the number of edges kept; src/dst hold nedges entries of room.     */
int64_t synth_rmat(uint64_t key, int scale, int64_t n, int64_t nedges,
                   double a, double b, double c, int32_t *src, int32_t *dst) {
    const uint32_t ta = (uint32_t)(a * 65536.0);
    const uint32_t tb = (uint32_t)((a + b) * 65536.0);
    const uint32_t tc = (uint32_t)((a + b + c) * 65536.0);
    const int words = (scale + 3) / 4;
    uint8_t *keep = (uint8_t *)malloc((size_t)(nedges > 0 ? nedges : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        int64_t s = 0, t = 0;
        for (int w = 0; w < words; ++w) {
            uint64_t r = sm_draw(key, (uint64_t)e * (uint64_t)words + (uint64_t)w);
            for (int q = 0; q < 4; ++q) {
                int l = w * 4 + q;
                if (l >= scale) break;
                uint32_t u = (uint32_t)((r >> (16 * q)) & 0xFFFFu);
                int sb = (u >= tb);                        /* quadrants c, d */
                int db = (u >= ta && u < tb) || (u >= tc); /* quadrants b, d */
                s |= (int64_t)sb << (scale - 1 - l);
                t |= (int64_t)db << (scale - 1 - l);
            }
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)t;
        keep[e] = (s < n && t < n);
    }
    int64_t out = 0;
    for (int64_t e = 0; e < nedges; ++e)
        if (keep[e]) { src[out] = src[e]; dst[out] = dst[e]; ++out; }
    free(keep);
    return out;
}

/* ------------------------------------------------------------------------ */
/* COO -> CSR with sorted, duplicate-free rows.                              */

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Builds CSR of an nrows x ncols pattern from ne (src, dst) pairs.
 * symmetrize: also insert (dst, src); drop_loops: drop src == dst.
 * colidx needs room for ne (2*ne when symmetrising) entries.  Returns nnz. */
int64_t synth_coo_to_csr(int64_t nrows, int64_t ne, const int32_t *src, const int32_t *dst,
                         int symmetrize, int drop_loops, int32_t *rowptr, int32_t *colidx) {
    int64_t *cnt = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
    for (int64_t e = 0; e < ne; ++e) {
        if (drop_loops && src[e] == dst[e]) continue;
        cnt[src[e] + 1]++;
        if (symmetrize) cnt[dst[e] + 1]++;
    }
    for (int64_t i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
    int64_t *pos = (int64_t *)malloc(((size_t)nrows + 1) * sizeof(int64_t));
    memcpy(pos, cnt, ((size_t)nrows + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < ne; ++e) {
        if (drop_loops && src[e] == dst[e]) continue;
        colidx[pos[src[e]]++] = dst[e];
        if (symmetrize) colidx[pos[dst[e]]++] = src[e];
    }
    /* sort and de-duplicate each row in place; keep row lengths in pos */
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nrows; ++i) {
        int32_t *r = colidx + cnt[i];
        int64_t len = cnt[i + 1] - cnt[i];
        if (len > 1) qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t t = 0; t < len; ++t)
            if (u == 0 || r[t] != r[u - 1]) r[u++] = r[t];
        pos[i] = u;
    }
    int64_t w = 0;
    rowptr[0] = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        int64_t len = pos[i];
        if (w != cnt[i]) memmove(colidx + w, colidx + cnt[i], (size_t)len * sizeof(int32_t));
        w += len;
        rowptr[i + 1] = (int32_t)w;
    }
    free(pos);
    free(cnt);
    return w;
}

/* ------------------------------------------------------------------------ */
/* Degree relabelling: new_id[v] = rank of v in order of non-increasing       */
/* degree, ties broken by ascending original id (Sec. 8.2).                  */

static const int32_t *g_deg_rowptr;
static int cmp_deg(const void *x, const void *y) {
    int32_t u = *(const int32_t *)x, v = *(const int32_t *)y;
    int32_t du = g_deg_rowptr[u + 1] - g_deg_rowptr[u];
    int32_t dv = g_deg_rowptr[v + 1] - g_deg_rowptr[v];
    if (du != dv) return (du < dv) ? 1 : -1;
    return (u > v) - (u < v);
}

void synth_degree_order(int64_t n, const int32_t *rowptr, int32_t *new_id) {
    int32_t *order = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v) order[v] = (int32_t)v;
    g_deg_rowptr = rowptr;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_deg);
    for (int64_t r = 0; r < n; ++r) new_id[order[r]] = (int32_t)r;
    free(order);
}

/* Relabels a pattern by new_id and emits COO pairs (new_i, new_j); when
 * strict_lower is set only pairs with new_j < new_i are kept.  Returns count. */
int64_t synth_relabel_coo(int64_t n, const int32_t *rowptr, const int32_t *colidx,
                          const int32_t *new_id, int strict_lower, int32_t *src, int32_t *dst) {
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t ni = new_id[i];
        for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            int32_t nj = new_id[colidx[t]];
            if (strict_lower && !(nj < ni)) continue;
            src[w] = ni;
            dst[w] = nj;
            ++w;
        }
    }
    return w;
}

/* ------------------------------------------------------------------------ */
/* Multi-source BFS frontier, two levels (input of one forward step of       */
/* batched betweenness centrality, Sec. 8.4).                                */

/* Picks nsrc distinct vertices of degree >= 1 from the key's stream. */
int64_t synth_pick_sources(uint64_t key, int64_t n, const int32_t *rowptr, int64_t nsrc, int32_t *out) {
    uint8_t *taken = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t got = 0, nonisolated = 0;
    for (int64_t v = 0; v < n; ++v) nonisolated += (rowptr[v + 1] > rowptr[v]);
    if (nsrc > nonisolated) nsrc = nonisolated;
    for (uint64_t t = 0; got < nsrc; ++t) {
        int64_t v = (int64_t)(sm_draw(key, t) % (uint64_t)n);
        if (taken[v] || rowptr[v + 1] == rowptr[v]) continue;
        taken[v] = 1;
        out[got++] = (int32_t)v;
    }
    free(taken);
    return got;
}

/* For source s: L0 = {s} (sigma 1), L1 = N(s) \ L0 (sigma 1),
 * L2 = N(L1) \ (L0 u L1) with sigma(v) = sum of sigma(u), u in L1 adjacent to v.
 * Frontier row s = L2 with sigma, sorted; visited row s = L0 u L1 u L2, sorted.
 * With fill == 0 only the per-row counts are written (f_rowptr[1..], v_rowptr[1..]
 * hold counts, then are prefix-summed); with fill == 1 the rows are written. */
void synth_bfs2(int64_t n, const int32_t *rowptr, const int32_t *colidx,
                int64_t nsrc, const int32_t *sources, int fill,
                int64_t *f_rowptr, int32_t *f_colidx, int64_t *f_sigma,
                int64_t *v_rowptr, int32_t *v_colidx) {
    if (!fill) { f_rowptr[0] = 0; v_rowptr[0] = 0; }
    #pragma omp parallel
    {
        int8_t *level = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
        int64_t *sigma = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        memset(level, -1, (size_t)n);
        int32_t *l1 = NULL, *l2 = NULL;
        int64_t cap1 = 0, cap2 = 0;
        #pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nsrc; ++q) {
            int32_t s = sources[q];
            int64_t n1 = 0, n2 = 0;
            level[s] = 0; sigma[s] = 1;
            int64_t d = rowptr[s + 1] - rowptr[s];
            if (d > cap1) { cap1 = d; l1 = (int32_t *)realloc(l1, (size_t)cap1 * sizeof(int32_t)); }
            for (int32_t t = rowptr[s]; t < rowptr[s + 1]; ++t) {
                int32_t v = colidx[t];
                if (level[v] != -1) continue;
                level[v] = 1; sigma[v] = 1; l1[n1++] = v;
            }
            for (int64_t a = 0; a < n1; ++a) {
                int32_t u = l1[a];
                for (int32_t t = rowptr[u]; t < rowptr[u + 1]; ++t) {
                    int32_t v = colidx[t];
                    if (level[v] == -1) {
                        level[v] = 2; sigma[v] = 0;
                        if (n2 == cap2) { cap2 = cap2 ? 2 * cap2 : 1024; l2 = (int32_t *)realloc(l2, (size_t)cap2 * sizeof(int32_t)); }
                        l2[n2++] = v;
                    }
                    if (level[v] == 2) sigma[v] += sigma[u];
                }
            }
            if (!fill) {
                f_rowptr[q + 1] = n2;
                v_rowptr[q + 1] = 1 + n1 + n2;
            } else {
                if (n2 > 1) qsort(l2, (size_t)n2, sizeof(int32_t), cmp_i32);
                int32_t *fr = f_colidx + f_rowptr[q];
                int64_t *fs = f_sigma + f_rowptr[q];
                for (int64_t a = 0; a < n2; ++a) { fr[a] = l2[a]; fs[a] = sigma[l2[a]]; }
                int32_t *vr = v_colidx + v_rowptr[q];
                int64_t w = 0;
                vr[w++] = s;
                for (int64_t a = 0; a < n1; ++a) vr[w++] = l1[a];
                for (int64_t a = 0; a < n2; ++a) vr[w++] = l2[a];
                qsort(vr, (size_t)w, sizeof(int32_t), cmp_i32);
            }
            level[s] = -1;
            for (int64_t a = 0; a < n1; ++a) level[l1[a]] = -1;
            for (int64_t a = 0; a < n2; ++a) level[l2[a]] = -1;
        }
        free(level); free(sigma); free(l1); free(l2);
    }
    if (!fill) {
        for (int64_t q = 0; q < nsrc; ++q) { f_rowptr[q + 1] += f_rowptr[q]; v_rowptr[q + 1] += v_rowptr[q]; }
    }
}
