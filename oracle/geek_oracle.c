/*
 * FP64 / exact-integer CPU oracle for GEEK's data transformation, SILK seeding
 * and one-pass assignment (Luo, Huang, Tung: "A Generic Distributed Clustering
 * Framework for Massive Data", Sect. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it; the library
 * never links, includes or calls anything here, and this file includes no
 * header of the library.
 *
 * Precision and order rules (the paper fixes none of them; each is a reading):
 *  - dot products: s = sum_j (double)a_j * (double)x_j, sequentially in j,
 *    each product rounded to double (exact for float inputs), no FMA
 *    (build with -ffp-contract=off);
 *  - E2LSH code = floor((s + (double)b) / w) with IEEE round-to-nearest
 *    add and divide;
 *  - squared Euclidean distance = sum_j ((double)x_j - c_j)^2, sequential in
 *    j, subtract, multiply and add each rounded separately;
 *  - centroid = (sum over members in ascending id of (double)x) / count;
 *  - ties in every argmin / argmax go to the smallest index.
 *
 * Every function returns 0 on success, 1 on invalid input, 5 on overflow.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_NOMEM = 2, ORC_OVERFLOW = 5 };

/* ------------------------------------------------------------------------ */
/* Hashing.                                                                  */
/* ------------------------------------------------------------------------ */

/* E2LSH, the function h_{a,b}(x) = floor((a.x + b)/w) that Sect. 3.1
 * (Remarks) names: codes[i*F + f] for every object i and function f. */
int orc_e2lsh(int64_t n, int32_t d, const float *x, int64_t ldx, int32_t F,
              const float *a, const float *b, double w, int32_t *codes)
{
    if (n < 0 || d <= 0 || F <= 0 || ldx < d || !(w > 0.0)) return ORC_INVALID;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        const float *xi = x + i * ldx;
        for (int32_t f = 0; f < F; f++) {
            const float *af = a + (int64_t)f * d;
            double s = 0.0;
            for (int32_t j = 0; j < d; j++) {
                double p = (double)af[j] * (double)xi[j];
                s = s + p;
            }
            double t = (s + (double)b[f]) / w;
            double fl = floor(t);
            if (!(fl >= -2147483648.0 && fl <= 2147483647.0)) { bad |= 1; continue; }
            codes[i * F + f] = (int32_t)fl;
        }
    }
    return bad ? ORC_OVERFLOW : ORC_OK;
}

/* QALSH projection values of Alg. 1 (Sect. 3.1, homogeneous dense data):
 * s[i*m + f] = a_f . x_i with the pinned FP64 dot product (products of the
 * float inputs, summed in j order, no fused multiply-add). */
int orc_qalsh(int64_t n, int32_t d, const float *x, int64_t ldx, int32_t m,
              const float *a, double *s)
{
    if (n < 0 || d <= 0 || m <= 0 || ldx < d) return ORC_INVALID;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        const float *xi = x + i * ldx;
        for (int32_t f = 0; f < m; f++) {
            const float *af = a + (int64_t)f * d;
            double acc = 0.0;
            for (int32_t j = 0; j < d; j++) {
                double p = (double)af[j] * (double)xi[j];
                acc = acc + p;
            }
            s[i * m + f] = acc;
        }
    }
    return ORC_OK;
}

/* Sign random projection (SimHash, cited in Sect. 1): bit = [a.x >= 0],
 * with the same pinned dot product; -0.0 counts as >= 0. */
int orc_srp(int64_t n, int32_t d, const float *x, int64_t ldx, int32_t F,
            const float *a, uint8_t *bits)
{
    if (n < 0 || d <= 0 || F <= 0 || ldx < d) return ORC_INVALID;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        const float *xi = x + i * ldx;
        for (int32_t f = 0; f < F; f++) {
            const float *af = a + (int64_t)f * d;
            double s = 0.0;
            for (int32_t j = 0; j < d; j++) {
                double p = (double)af[j] * (double)xi[j];
                s = s + p;
            }
            bits[i * F + f] = (uint8_t)(s >= 0.0);
        }
    }
    return ORC_OK;
}

/* The random permutation pi of MinHash (Eq. 2) is realised by Dietzfelbinger's
 * multiply-add-shift hash: h(x) = floor(((A*x + B) mod 2^64) / 2^32). */
uint32_t orc_hash32(uint64_t A, uint64_t B, uint32_t x)
{
    uint64_t v = A * (uint64_t)x + B; /* unsigned arithmetic wraps mod 2^64 */
    return (uint32_t)(v >> 32);
}

/* MinHash (Eq. 2) of every set of a CSR collection under F hash functions:
 * out[i*F + f] = min over items a of set i of h_f(a).  An empty set gets
 * 0xFFFFFFFF (the paper does not define it). */
int orc_minhash_csr(int64_t n, const int64_t *off, const uint32_t *items, int32_t F,
                    const uint64_t *A, const uint64_t *B, uint32_t *out)
{
    if (n < 0 || F <= 0) return ORC_INVALID;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        for (int32_t f = 0; f < F; f++) {
            uint32_t m = 0xFFFFFFFFu;
            for (int64_t p = off[i]; p < off[i + 1]; p++) {
                uint32_t h = orc_hash32(A[f], B[f], items[p]);
                if (h < m) m = h;
            }
            out[i * F + f] = m;
        }
    }
    return ORC_OK;
}

/* DOPH reduction of the sparse transform (Alg. 3, first step; densified
 * one permutation hashing with rotation).  One hash pi(v) = h(Ap, Bp, v)
 * stands for the permutation; the hash range is cut into Dp equal bins:
 * bin(v) = (pi(v) * Dp) >> 32, offset(v) = (pi(v) * Dp) mod 2^32.  Bin b
 * keeps the smallest offset of its items; an empty bin b borrows the value
 * of the first non-empty bin b + t (t >= 1, circular) and records t.  An
 * empty set: t = Dp, value 2^32 - 1 everywhere.  Token of bin b:
 * (b << 48) | (t << 32) | value, so the reduced object is a set of Dp
 * distinct 64-bit tokens.  Dp <= 65535. */
int orc_doph(int64_t n, const int64_t *off, const uint32_t *items, int32_t Dp, uint64_t Ap, uint64_t Bp,
             uint64_t *tokens)
{
    if (n < 0 || Dp < 1 || Dp > 65535) return ORC_INVALID;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        uint64_t *m = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)Dp);
        if (!m) { bad |= 1; continue; }
        for (int32_t b = 0; b < Dp; b++) m[b] = UINT64_MAX; /* empty */
        for (int64_t p = off[i]; p < off[i + 1]; p++) {
            uint64_t scaled = (uint64_t)orc_hash32(Ap, Bp, items[p]) * (uint64_t)Dp;
            int32_t b = (int32_t)(scaled >> 32);
            uint64_t o = scaled & 0xFFFFFFFFull;
            if (o < m[b]) m[b] = o;
        }
        for (int32_t b = 0; b < Dp; b++) {
            uint64_t t = 0, v = m[b];
            while (v == UINT64_MAX && t < (uint64_t)Dp) {
                t++;
                v = m[(b + t) % Dp];
            }
            if (v == UINT64_MAX) { t = (uint64_t)Dp; v = 0xFFFFFFFFull; }
            tokens[i * Dp + b] = ((uint64_t)b << 48) | (t << 32) | v;
        }
        free(m);
    }
    return bad ? ORC_INVALID : ORC_OK;
}

/* MinHash of fixed-length rows of 64-bit tokens: h(A, B, x) =
 * ((A x + B) mod 2^64) >> 32 with the full 64-bit token x. */
int orc_minhash_rows64(int64_t n, int32_t m, const uint64_t *tokens, int32_t F, const uint64_t *A,
                       const uint64_t *B, uint32_t *out)
{
    if (n < 0 || m < 0 || F <= 0) return ORC_INVALID;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int32_t f = 0; f < F; f++) {
            uint32_t best = 0xFFFFFFFFu;
            for (int32_t j = 0; j < m; j++) {
                uint32_t h = (uint32_t)((A[f] * tokens[i * m + j] + B[f]) >> 32);
                if (h < best) best = h;
            }
            out[i * F + f] = best;
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* A stable sort of row indices by lexicographic int64 keys (a library-style */
/* primitive: parallel merge sort; equal keys keep ascending index).         */
/* ------------------------------------------------------------------------ */

static inline int row_less(const int64_t *keys, int32_t W, int32_t a, int32_t b)
{
    const int64_t *ka = keys + (int64_t)a * W, *kb = keys + (int64_t)b * W;
    for (int32_t w = 0; w < W; w++) {
        if (ka[w] < kb[w]) return 1;
        if (ka[w] > kb[w]) return 0;
    }
    return 0;
}

static void merge_runs(const int64_t *keys, int32_t W, const int32_t *src, int32_t *dst,
                       int64_t lo, int64_t mid, int64_t hi)
{
    int64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        /* take from the right run only when strictly smaller: stability */
        if (row_less(keys, W, src[j], src[i])) dst[o++] = src[j++];
        else dst[o++] = src[i++];
    }
    while (i < mid) dst[o++] = src[i++];
    while (j < hi) dst[o++] = src[j++];
}

static void msort_seq(const int64_t *keys, int32_t W, int32_t *a, int32_t *tmp, int64_t lo, int64_t hi)
{
    /* bottom-up; result ends in a[lo..hi) */
    int64_t n = hi - lo;
    int32_t *src = a, *dst = tmp;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t s = lo; s < hi; s += 2 * width) {
            int64_t m = s + width < hi ? s + width : hi;
            int64_t e = s + 2 * width < hi ? s + 2 * width : hi;
            merge_runs(keys, W, src, dst, s, m, e);
        }
        int32_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a + lo, src + lo, (size_t)n * sizeof(int32_t));
}

/* perm := indices 0..n-1 stably sorted by keys[i*W .. i*W+W) */
int orc_sort_rows(int64_t n, int32_t W, const int64_t *keys, int32_t *perm)
{
    if (n < 0 || n > 2147483647LL || W <= 0) return ORC_INVALID;
    int32_t *tmp = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!tmp) return ORC_NOMEM;
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    int T = 1;
#ifdef _OPENMP
    T = omp_get_max_threads();
#endif
    int chunks = 1;
    while (chunks < T && chunks < 64) chunks *= 2;
    if (n < 65536) chunks = 1;
    int64_t *bound = (int64_t *)malloc(sizeof(int64_t) * (chunks + 1));
    for (int c = 0; c <= chunks; c++) bound[c] = n * c / chunks;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < chunks; c++) msort_seq(keys, W, perm, tmp, bound[c], bound[c + 1]);
    int32_t *src = perm, *dst = tmp;
    for (int step = 1; step < chunks; step *= 2) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < chunks; c += 2 * step) {
            int64_t lo = bound[c], mid = bound[c + step < chunks ? c + step : chunks];
            int64_t hi = bound[c + 2 * step < chunks ? c + 2 * step : chunks];
            merge_runs(keys, W, src, dst, lo, mid, hi);
        }
        int32_t *t = src; src = dst; dst = t;
    }
    if (src != perm) memcpy(perm, src, (size_t)n * sizeof(int32_t));
    free(bound);
    free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Bucketing: the static (K,L) framework of Sect. 2.2 and Algs. 2-3.         */
/* ------------------------------------------------------------------------ */

/* Group every table's objects by their K-word key (T[G(x_j)].push(j) in
 * Algs. 2-3).  keys is [L][n][W] int64.  Canonical bucket id of object i in
 * table l = rank of its key among the table's distinct keys in ascending
 * lexicographic order.  members[l][*] lists object ids by (bucket, id);
 * bucket_off[l][0..n_buckets[l]] are the bucket boundaries in it. */
int orc_group(int64_t n, int32_t L, int32_t W, const int64_t *keys,
              int32_t *obj_bucket, int64_t *n_buckets, int32_t *members, int64_t *bucket_off)
{
    if (n < 0 || n > 2147483647LL || L <= 0 || W <= 0) return ORC_INVALID;
    for (int32_t l = 0; l < L; l++) {
        const int64_t *kl = keys + (int64_t)l * n * W;
        int32_t *perm = members + (int64_t)l * n;
        int rc = orc_sort_rows(n, W, kl, perm);
        if (rc) return rc;
        int64_t *bo = bucket_off + (int64_t)l * (n + 1);
        int32_t *ob = obj_bucket + (int64_t)l * n;
        int64_t nb = 0;
        for (int64_t p = 0; p < n; p++) {
            int new_bucket = (p == 0) ||
                             memcmp(kl + (int64_t)perm[p] * W, kl + (int64_t)perm[p - 1] * W,
                                    sizeof(int64_t) * W) != 0;
            if (new_bucket) bo[nb++] = p;
            ob[perm[p]] = (int32_t)(nb - 1);
        }
        bo[nb] = n;
        n_buckets[l] = nb;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SILK (Alg. 4).                                                            */
/* ------------------------------------------------------------------------ */

/* Bucket signatures: sig[g*nf + f] = min over members of bucket g of h_f(id),
 * the MinHash of a bucket viewed as a set of object ids (Alg. 4, G(B_j)). */
int orc_bucket_sigs(int64_t NB, const int64_t *boff, const int32_t *bmem, int32_t nf,
                    const uint64_t *A, const uint64_t *B, uint32_t *sig)
{
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t g = 0; g < NB; g++) {
        for (int32_t f = 0; f < nf; f++) {
            uint32_t m = 0xFFFFFFFFu;
            for (int64_t p = boff[g]; p < boff[g + 1]; p++) {
                uint32_t h = orc_hash32(A[f], B[f], (uint32_t)bmem[p]);
                if (h < m) m = h;
            }
            sig[g * nf + f] = m;
        }
    }
    return ORC_OK;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Majority voting (Sect. 3.2): the objects that occur in more than half of
 * the nb buckets listed in bin[0..nb), i.e. 2*cnt > nb, ascending.  Writes
 * them to out (capacity: total members) and returns the count. */
static int64_t vote_one(int32_t nb, const int64_t *bin, const int64_t *boff, const int32_t *bmem,
                        int32_t *scratch, int32_t *out)
{
    int64_t tot = 0;
    for (int32_t b = 0; b < nb; b++) {
        int64_t g = bin[b];
        for (int64_t p = boff[g]; p < boff[g + 1]; p++) scratch[tot++] = bmem[p];
    }
    qsort(scratch, (size_t)tot, sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t p = 0; p < tot;) {
        int64_t q = p;
        while (q < tot && scratch[q] == scratch[p]) q++;
        if (2 * (q - p) > nb) out[k++] = scratch[p];
        p = q;
    }
    return k;
}

/* Exposed for tests: majority vote over explicit bins (each bin a list of
 * bucket ids).  Bins with at most one bucket are skipped, as in Alg. 4;
 * a kept set must have at least delta objects.  out_off[b] / out_ids give
 * each bin's C_shared (empty when skipped or below delta). */
int orc_vote_bins(int64_t nbins, const int64_t *bin_off, const int64_t *bin_bucket,
                  const int64_t *boff, const int32_t *bmem, int32_t delta,
                  int64_t *out_off, int32_t *out_ids)
{
    int64_t cap = 0;
    for (int64_t b = 0; b < nbins; b++) {
        int64_t t = 0;
        for (int64_t q = bin_off[b]; q < bin_off[b + 1]; q++) t += boff[bin_bucket[q] + 1] - boff[bin_bucket[q]];
        if (t > cap) cap = t;
    }
    int32_t *scr = (int32_t *)malloc(sizeof(int32_t) * (cap + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (cap + 1));
    out_off[0] = 0;
    for (int64_t b = 0; b < nbins; b++) {
        int32_t nb = (int32_t)(bin_off[b + 1] - bin_off[b]);
        int64_t k = 0;
        if (nb > 1) {
            k = vote_one(nb, bin_bucket + bin_off[b], boff, bmem, scr, tmp);
            if (k < delta) k = 0;
            memcpy(out_ids + out_off[b], tmp, sizeof(int32_t) * k);
        }
        out_off[b + 1] = out_off[b] + k;
    }
    free(scr);
    free(tmp);
    return ORC_OK;
}

/* growable CSR list of sets */
typedef struct { int64_t n, cap_sets, nids, cap_ids; int64_t *off; int32_t *ids; } setlist;

static int sl_init(setlist *s)
{
    s->n = 0; s->cap_sets = 1024; s->nids = 0; s->cap_ids = 1 << 16;
    s->off = (int64_t *)malloc(sizeof(int64_t) * (s->cap_sets + 1));
    s->ids = (int32_t *)malloc(sizeof(int32_t) * s->cap_ids);
    if (!s->off || !s->ids) return ORC_NOMEM;
    s->off[0] = 0;
    return ORC_OK;
}
static int sl_push(setlist *s, const int32_t *ids, int64_t k)
{
    if (s->n + 1 > s->cap_sets) {
        s->cap_sets *= 2;
        s->off = (int64_t *)realloc(s->off, sizeof(int64_t) * (s->cap_sets + 1));
        if (!s->off) return ORC_NOMEM;
    }
    while (s->nids + k > s->cap_ids) {
        s->cap_ids *= 2;
        s->ids = (int32_t *)realloc(s->ids, sizeof(int32_t) * s->cap_ids);
        if (!s->ids) return ORC_NOMEM;
    }
    memcpy(s->ids + s->nids, ids, sizeof(int32_t) * k);
    s->nids += k;
    s->n++;
    s->off[s->n] = s->nids;
    return ORC_OK;
}

/* canonical order of seeds: lexicographic on the ascending member lists, a
 * proper prefix first */
static int set_cmp(const int32_t *a, int64_t na, const int32_t *b, int64_t nb)
{
    int64_t m = na < nb ? na : nb;
    for (int64_t i = 0; i < m; i++) {
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    }
    return (na > nb) - (na < nb);
}

static const setlist *g_sort_sl; /* qsort context for set ordering (single-threaded use) */
static int cmp_set_idx(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    const setlist *s = g_sort_sl;
    int c = set_cmp(s->ids + s->off[a], s->off[a + 1] - s->off[a], s->ids + s->off[b], s->off[b + 1] - s->off[b]);
    if (c) return c;
    return (a > b) - (a < b);
}

/* Near-duplicate removal (Sect. 3.2, "repeat the procedure with L = 1") on
 * given bins of the seed multiset C (CSR coff/cids; bin b lists the sets
 * bin_set[bin_off[b] .. bin_off[b+1])):
 *   - a bin holding one set keeps it (Example 2 keeps four distinct seeds,
 *     which the skip of single-bucket bins would otherwise delete),
 *   - a bin holding several sets yields their majority-vote set when its
 *     size is >= delta, otherwise its member smallest in canonical order;
 * then exact duplicates are dropped and the seeds sorted in canonical order
 * (lexicographic on ascending member lists).  Returns a malloc'd CSR. */
int orc_dedup_bins(int64_t nC, const int64_t *coff, const int32_t *cids, int64_t nbins,
                   const int64_t *bin_off, const int64_t *bin_set, int32_t delta,
                   int64_t *k_out, int64_t **seed_off, int32_t **seed_ids)
{
    setlist D;
    if (sl_init(&D)) return ORC_NOMEM;
    int64_t cap = 1;
    for (int64_t i = 0; i < nC; i++) cap += coff[i + 1] - coff[i];
    int32_t *scr = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * cap);
    if (!scr || !out) return ORC_NOMEM;
    for (int64_t bi = 0; bi < nbins; bi++) {
        const int64_t *bl = bin_set + bin_off[bi];
        int32_t nb = (int32_t)(bin_off[bi + 1] - bin_off[bi]);
        if (nb <= 0) continue;
        if (nb == 1) {
            int64_t s = bl[0];
            if (sl_push(&D, cids + coff[s], coff[s + 1] - coff[s])) return ORC_NOMEM;
            continue;
        }
        int64_t k = vote_one(nb, bl, coff, cids, scr, out);
        if (k >= delta) {
            if (sl_push(&D, out, k)) return ORC_NOMEM;
        } else {
            int64_t best = bl[0];
            for (int32_t b = 1; b < nb; b++) {
                int64_t s = bl[b];
                if (set_cmp(cids + coff[s], coff[s + 1] - coff[s], cids + coff[best],
                            coff[best + 1] - coff[best]) < 0)
                    best = s;
            }
            if (sl_push(&D, cids + coff[best], coff[best + 1] - coff[best])) return ORC_NOMEM;
        }
    }
    free(scr);
    free(out);

    /* exact duplicates out, canonical order */
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(D.n > 0 ? D.n : 1));
    for (int64_t i = 0; i < D.n; i++) idx[i] = i;
    g_sort_sl = &D;
    qsort(idx, (size_t)D.n, sizeof(int64_t), cmp_set_idx);
    setlist E;
    if (sl_init(&E)) return ORC_NOMEM;
    for (int64_t r = 0; r < D.n; r++) {
        int64_t s = idx[r];
        if (r > 0) {
            int64_t t = idx[r - 1];
            if (set_cmp(D.ids + D.off[s], D.off[s + 1] - D.off[s], D.ids + D.off[t], D.off[t + 1] - D.off[t]) == 0)
                continue;
        }
        if (sl_push(&E, D.ids + D.off[s], D.off[s + 1] - D.off[s])) return ORC_NOMEM;
    }
    free(idx); free(D.off); free(D.ids);
    *k_out = E.n;
    *seed_off = E.off;
    *seed_ids = E.ids;
    return ORC_OK;
}

/* SILK, Alg. 4, on the collection of buckets (CSR boff/bmem; bucket g holds
 * object ids in ascending order).  For each of the Ls SILK tables the Ks
 * hashes mh_a/mh_b[t*Ks + k] group buckets into bins; bins holding at most
 * one bucket are skipped; every other bin contributes its majority-vote set
 * C_shared when |C_shared| >= delta.  Near-duplicates are then removed by
 * one more pass with a single table of Ks fresh hashes dd_a/dd_b:
 *   - a bin holding one set keeps it (Example 2 keeps four distinct seeds),
 *   - a bin holding several sets yields their majority-vote set when its
 *     size is >= delta, otherwise its member smallest in canonical order;
 * exact duplicates are dropped and seeds sorted in canonical order.  The
 * result is a malloc'd CSR (free with orc_free). */
int orc_silk(int64_t NB, const int64_t *boff, const int32_t *bmem, int32_t Ks, int32_t Ls,
             int32_t delta, const uint64_t *mh_a, const uint64_t *mh_b, const uint64_t *dd_a,
             const uint64_t *dd_b, int64_t *k_out, int64_t **seed_off, int32_t **seed_ids,
             int64_t *n_multiset)
{
    if (NB < 0 || Ks <= 0 || Ls <= 0 || delta < 1) return ORC_INVALID;
    setlist C;
    if (sl_init(&C)) return ORC_NOMEM;
    int64_t maxb = 0;
    for (int64_t g = 0; g < NB; g++) if (boff[g + 1] - boff[g] > maxb) maxb = boff[g + 1] - boff[g];

    uint32_t *sig = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(NB > 0 ? NB : 1) * Ks);
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NB > 0 ? NB : 1) * Ks);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(NB > 0 ? NB : 1));
    int64_t *binb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NB > 0 ? NB : 1));
    if (!sig || !key || !perm || !binb) return ORC_NOMEM;

    for (int32_t t = 0; t < Ls; t++) {
        orc_bucket_sigs(NB, boff, bmem, Ks, mh_a + (int64_t)t * Ks, mh_b + (int64_t)t * Ks, sig);
        for (int64_t i = 0; i < NB * Ks; i++) key[i] = (int64_t)sig[i];
        int rc = orc_sort_rows(NB, Ks, key, perm);
        if (rc) return rc;
        /* bins = runs of equal signatures; list bin starts */
        int64_t nbins = 0;
        int64_t *starts = binb; /* reuse: starts of runs in perm order */
        for (int64_t p = 0; p < NB; p++) {
            if (p == 0 || memcmp(key + (int64_t)perm[p] * Ks, key + (int64_t)perm[p - 1] * Ks,
                                 sizeof(int64_t) * Ks) != 0)
                starts[nbins++] = p;
        }
        /* vote every bin with >= 2 buckets, in parallel, collecting per bin */
        int64_t *res_off = (int64_t *)calloc((size_t)nbins + 1, sizeof(int64_t));
        int32_t **res = (int32_t **)calloc((size_t)(nbins > 0 ? nbins : 1), sizeof(int32_t *));
#pragma omp parallel
        {
            int32_t *scr = NULL, *out = NULL;
            int64_t cap = 0;
#pragma omp for schedule(dynamic, 256)
            for (int64_t bi = 0; bi < nbins; bi++) {
                int64_t s = starts[bi], e = (bi + 1 < nbins) ? starts[bi + 1] : NB;
                int32_t nb = (int32_t)(e - s);
                if (nb <= 1) continue; /* isolated bucket: ignored (Alg. 4) */
                int64_t tot = 0;
                int64_t *bl = (int64_t *)malloc(sizeof(int64_t) * nb);
                for (int32_t b = 0; b < nb; b++) {
                    bl[b] = perm[s + b];
                    tot += boff[bl[b] + 1] - boff[bl[b]];
                }
                if (tot > cap) {
                    cap = tot;
                    scr = (int32_t *)realloc(scr, sizeof(int32_t) * cap);
                    out = (int32_t *)realloc(out, sizeof(int32_t) * cap);
                }
                int64_t k = vote_one(nb, bl, boff, bmem, scr, out);
                free(bl);
                if (k >= delta) {
                    res[bi] = (int32_t *)malloc(sizeof(int32_t) * k);
                    memcpy(res[bi], out, sizeof(int32_t) * k);
                    res_off[bi] = k;
                }
            }
            free(scr);
            free(out);
        }
        for (int64_t bi = 0; bi < nbins; bi++) {
            if (res[bi]) {
                if (sl_push(&C, res[bi], res_off[bi])) return ORC_NOMEM;
                free(res[bi]);
            }
        }
        free(res);
        free(res_off);
    }
    free(sig); free(key); free(perm); free(binb);
    *n_multiset = C.n;

    /* --- near-duplicate removal: one more pass with L = 1 over C --- */
    int64_t nC = C.n;
    uint32_t *csig = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nC > 0 ? nC : 1) * Ks);
    int64_t *ckey = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nC > 0 ? nC : 1) * Ks);
    int32_t *cperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nC > 0 ? nC : 1));
    int64_t *cbin_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nC + 1));
    int64_t *cbin_set = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nC > 0 ? nC : 1));
    if (!csig || !ckey || !cperm || !cbin_off || !cbin_set) return ORC_NOMEM;
    orc_bucket_sigs(nC, C.off, C.ids, Ks, dd_a, dd_b, csig);
    for (int64_t i = 0; i < nC * Ks; i++) ckey[i] = (int64_t)csig[i];
    int rc = orc_sort_rows(nC, Ks, ckey, cperm);
    if (rc) return rc;
    int64_t nbins = 0;
    for (int64_t p = 0; p < nC; p++) {
        if (p == 0 || memcmp(ckey + (int64_t)cperm[p] * Ks, ckey + (int64_t)cperm[p - 1] * Ks,
                             sizeof(int64_t) * Ks) != 0)
            cbin_off[nbins++] = p;
        cbin_set[p] = cperm[p];
    }
    cbin_off[nbins] = nC;
    rc = orc_dedup_bins(nC, C.off, C.ids, nbins, cbin_off, cbin_set, delta, k_out, seed_off, seed_ids);
    free(csig); free(ckey); free(cperm); free(cbin_off); free(cbin_set);
    free(C.off); free(C.ids);
    return rc;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Data assignment (Sect. 3.3) and the central vectors.                      */
/* ------------------------------------------------------------------------ */

/* Centroid of every seed: FP64 sum over members in ascending id, then one
 * IEEE division by the member count. */
int orc_centroids(int64_t n, int32_t d, const float *x, int64_t ldx, int64_t k,
                  const int64_t *soff, const int32_t *sids, double *c)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < k; j++) {
        int64_t cnt = soff[j + 1] - soff[j];
        for (int32_t t = 0; t < d; t++) {
            double s = 0.0;
            for (int64_t p = soff[j]; p < soff[j + 1]; p++) s = s + (double)x[(int64_t)sids[p] * ldx + t];
            c[j * d + t] = s / (double)cnt;
        }
    }
    (void)n;
    return ORC_OK;
}

/* Eq. 1 with squared Euclidean distance: label = argmin_j sum_t (x_t - c_jt)^2,
 * ties to the smallest j; dist receives that minimum.  k == 0 gives -1. */
int orc_assign_dense(int64_t n, int32_t d, const float *x, int64_t ldx, int64_t k,
                     const double *c, int32_t *labels, double *dist)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double best = INFINITY;
        int32_t bj = -1;
        const float *xi = x + i * ldx;
        for (int64_t j = 0; j < k; j++) {
            const double *cj = c + j * d;
            double D = 0.0;
            for (int32_t t = 0; t < d; t++) {
                double e = (double)xi[t] - cj[t];
                double q = e * e;
                D = D + q;
            }
            if (D < best) { best = D; bj = (int32_t)j; }
        }
        labels[i] = bj;
        dist[i] = best;
    }
    return ORC_OK;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Mode of every categorical attribute over each seed's members (Sect. 3.3,
 * "mode" central vector): the most frequent value, ties to the smallest. */
int orc_modes(int64_t n, int32_t A, const int64_t *attrs, int64_t k, const int64_t *soff,
              const int32_t *sids, int64_t *modes)
{
    (void)n;
#pragma omp parallel
    {
        int64_t *buf = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < k; j++) {
            int64_t cnt = soff[j + 1] - soff[j];
            if (cnt > cap) { cap = cnt; buf = (int64_t *)realloc(buf, sizeof(int64_t) * cap); }
            for (int32_t a = 0; a < A; a++) {
                for (int64_t p = 0; p < cnt; p++) buf[p] = attrs[(int64_t)sids[soff[j] + p] * A + a];
                qsort(buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
                int64_t bestv = buf[0], bestc = 0;
                for (int64_t p = 0; p < cnt;) {
                    int64_t q = p;
                    while (q < cnt && buf[q] == buf[p]) q++;
                    if (q - p > bestc) { bestc = q - p; bestv = buf[p]; } /* ascending: first max wins */
                    p = q;
                }
                modes[j * A + a] = bestv;
            }
        }
        free(buf);
    }
    return ORC_OK;
}

/* Assignment with Dist = 1 - Jaccard on attribute-tagged values (Sect. 2.1):
 * for A attributes Jaccard = m / (2A - m) with m the matching attributes, so
 * the closest mode maximises m; ties to the smallest j. */
int orc_assign_cat(int64_t n, int32_t A, const int64_t *attrs, int64_t k, const int64_t *modes,
                   int32_t *labels, int32_t *matches)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int32_t bm = -1, bj = -1;
        for (int64_t j = 0; j < k; j++) {
            int32_t m = 0;
            for (int32_t a = 0; a < A; a++) m += attrs[i * A + a] == modes[j * A + a];
            if (m > bm) { bm = m; bj = (int32_t)j; }
        }
        labels[i] = bj;
        matches[i] = bm;
    }
    return ORC_OK;
}

/* Sparse central vector: the items present in more than half of the seed's
 * member sets (the binary mode per dimension).  Returns a malloc'd CSR. */
int orc_sparse_centres(const int64_t *off, const uint32_t *items, int64_t k, const int64_t *soff,
                       const int32_t *sids, int64_t **coff_out, uint32_t **citems_out)
{
    int64_t *coff = (int64_t *)malloc(sizeof(int64_t) * (k + 1));
    uint32_t **parts = (uint32_t **)calloc((size_t)(k > 0 ? k : 1), sizeof(uint32_t *));
    int64_t *plen = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < k; j++) {
        int64_t cnt = soff[j + 1] - soff[j], tot = 0;
        for (int64_t p = soff[j]; p < soff[j + 1]; p++) tot += off[sids[p] + 1] - off[sids[p]];
        int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (tot > 0 ? tot : 1));
        int64_t q = 0;
        for (int64_t p = soff[j]; p < soff[j + 1]; p++)
            for (int64_t r = off[sids[p]]; r < off[sids[p] + 1]; r++) buf[q++] = items[r];
        qsort(buf, (size_t)tot, sizeof(int64_t), cmp_i64);
        uint32_t *res = (uint32_t *)malloc(sizeof(uint32_t) * (tot > 0 ? tot : 1));
        int64_t m = 0;
        for (int64_t p = 0; p < tot;) {
            int64_t e = p;
            while (e < tot && buf[e] == buf[p]) e++;
            if (2 * (e - p) > cnt) res[m++] = (uint32_t)buf[p];
            p = e;
        }
        free(buf);
        parts[j] = res;
        plen[j] = m;
    }
    coff[0] = 0;
    for (int64_t j = 0; j < k; j++) coff[j + 1] = coff[j] + plen[j];
    uint32_t *ci = (uint32_t *)malloc(sizeof(uint32_t) * (coff[k] > 0 ? coff[k] : 1));
    for (int64_t j = 0; j < k; j++) {
        memcpy(ci + coff[j], parts[j], sizeof(uint32_t) * plen[j]);
        free(parts[j]);
    }
    free(parts);
    free(plen);
    *coff_out = coff;
    *citems_out = ci;
    return ORC_OK;
}

/* Assignment with Dist = 1 - Jaccard between sets (Sect. 2.1, Eq. 1): the
 * label maximises |A n C| / |A u C|, compared exactly as fractions by 64-bit
 * cross-multiplication; an empty union counts as similarity 0; ties go to
 * the smallest j.  Both item lists must be ascending. */
int orc_assign_jaccard(int64_t n, const int64_t *off, const uint32_t *items, int64_t k,
                       const int64_t *coff, const uint32_t *citems, int32_t *labels,
                       int64_t *inter_out, int64_t *union_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        int64_t bn = -1, bd = 1;
        int32_t bj = -1;
        const uint32_t *a = items + off[i];
        int64_t na = off[i + 1] - off[i];
        for (int64_t j = 0; j < k; j++) {
            const uint32_t *c = citems + coff[j];
            int64_t nc = coff[j + 1] - coff[j], p = 0, q = 0, in = 0;
            while (p < na && q < nc) {
                if (a[p] == c[q]) { in++; p++; q++; }
                else if (a[p] < c[q]) p++;
                else q++;
            }
            int64_t un = na + nc - in;
            int64_t num = un ? in : 0, den = un ? un : 1;
            if (bj < 0 || num * bd > bn * den) { bn = num; bd = den; bj = (int32_t)j; }
        }
        labels[i] = bj;
        inter_out[i] = bn;
        union_out[i] = bd;
    }
    return ORC_OK;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
