// SILK seeding (Sect. 3.2, Alg. 4) on the device.
//
// The buckets of all transform tables become virtual buckets (identical
// one-object buckets merged, with a weight).  For each SILK table: the
// MinHash signature of every virtual bucket, bins = groups of equal
// signatures found by hashing (seen-once / seen-twice maps, then
// fingerprinted grouping tables; one-object buckets joined to a group by a
// claim where a one-to-one MinHash function makes that exact), majority
// voting by sorting (bin, id) pairs and counting runs, the delta filter, then
// compaction into a CSR multiset.  The near-duplicate removal pass groups the
// multiset's sets by sorted signatures, followed by a canonical lexicographic
// sort and removal of exact duplicates.
#include "internal.cuh"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 finalizer (Steele, Lea and Flood, 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// 64-bit hash of a signature (lo, hi) of instance tg: slot index (low
// bits) and fingerprint (high word) of the grouping tables
__device__ __forceinline__ uint64_t sig_hash(uint64_t lo, uint64_t hi, uint32_t tg) {
    return mix64(lo ^ mix64(hi + 0x9e3779b97f4a7c15ull * (uint64_t)(tg + 1)));
}

// Sets seen once / twice: two bitmaps with a part of seen_mask + 1 bits per
// table (part t at t * (seen_mask + 1)), indexed by a hash of the signature
// hash.  A set whose bit in the second map is clear has no other set with
// its signature in its table: its bin holds it alone, and it skips the
// grouping table.  Blocks run roughly table by table, so the part in use
// stays in L2.
__device__ __forceinline__ uint64_t seen_pos(uint64_t hf, int t, uint64_t seen_mask) {
    return (uint64_t)t * (seen_mask + 1) + (mix64(hf ^ 0xd1b54a32d192ed03ull) & seen_mask);
}

// signature key of set g under Ks functions (first function most
// significant): Ks <= 2 fits the low word, Ks 3..4 use the high word too.
// Batched instances (count > 1): ids are global rows, instance i owning
// [row_off[i], row_off[i + 1]); a set lies inside one instance, whose
// coefficients (A/B + i * coef_stride) hash its local ids, and tag[g] = i.
// (set_inst, when given, holds every set's instance: no search per set)
__global__ void k_set_sig(int64_t nsets, const int64_t *__restrict__ soff,
                          const uint32_t *__restrict__ sids, int Ks, const uint64_t *__restrict__ A,
                          const uint64_t *__restrict__ B, const int64_t *__restrict__ row_off, int count,
                          const uint32_t *__restrict__ set_inst, int64_t coef_stride, uint64_t *__restrict__ klo,
                          uint64_t *__restrict__ khi, uint32_t *__restrict__ vals, uint32_t *__restrict__ tag) {
    // blockIdx.y = SILK table of this segment (functions t*Ks .. t*Ks+Ks-1)
    const int t = blockIdx.y;
    const int64_t so = (int64_t)t * nsets;
    uint64_t a[4], b[4];
    for (int k = 0; k < Ks; k++) {
        a[k] = A[t * Ks + k];
        b[k] = B[t * Ks + k];
    }
    int have = count > 1 ? -1 : 0;  // instance whose coefficients are in a / b
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nsets;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s0 = soff[g], s1 = soff[g + 1];
        int inst = 0;
        uint32_t base = 0;
        if (count > 1 && s1 > s0) {
            inst = set_inst ? (int)set_inst[g] : find_inst(row_off, count, (int64_t)sids[s0]);
            base = (uint32_t)row_off[inst];
            if (inst != have) {
                for (int k = 0; k < Ks; k++) {
                    a[k] = A[inst * coef_stride + t * Ks + k];
                    b[k] = B[inst * coef_stride + t * Ks + k];
                }
                have = inst;
            }
        }
        uint32_t m[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
        for (int64_t p = s0; p < s1; p++) {
            const uint32_t id = sids[p] - base;
            for (int k = 0; k < Ks; k++) m[k] = min(m[k], mh_hash32(a[k], b[k], id));
        }
        uint64_t hi = 0, lo = 0;
        for (int k = 0; k < Ks; k++) {
            hi = (hi << 32) | (lo >> 32);
            lo = (lo << 32) | m[k];
        }
        klo[so + g] = lo;
        if (khi) khi[so + g] = hi;
        if (vals) vals[so + g] = (uint32_t)g;
        if (tag) tag[so + g] = (uint32_t)inst;
    }
}

// The signatures of sets g0 .. nsets-1 (as k_set_sig; set_inst required for
// batched instances) for the grouping tables, with the seen-once /
// seen-twice marks: a set marks its position (a hash of signature and
// instance) in the seen-once map and, when the bit was already set, in the
// seen-twice map.
//
// With ms given, sets 0 .. g0-1 are the one-object virtual buckets and
// function kst[instance * kst_stride + t] of the table is injective on the
// instance's ids (k_mh_injective).  Set B then shares its signature with the
// one-object bucket {a} exactly when a is B's argmin under that function
// (unique, the function being injective), a attains B's minimum under every
// other function too, and a has a one-object bucket (single_of): the
// injective component forces a to be that argmin, and the others then agree.
// ms[t * (nsets - g0) + g - g0] receives that bucket (or -1), and a set with
// one marks the seen-twice map directly (its bin holds two sets).
//
// A thread takes SM_U sets at a time, loads their bounds and first two
// members together, and issues the seen-once atomics of all SM_U sets before
// it waits for any of them.
constexpr int SM_U = 4;
__global__ void __launch_bounds__(256, 3)
    k_set_sig_marks(int64_t nsets, const int64_t *__restrict__ soff, const uint32_t *__restrict__ sids, int Ks,
                    const uint64_t *__restrict__ A, const uint64_t *__restrict__ B,
                    const int64_t *__restrict__ row_off, int count, const uint32_t *__restrict__ set_inst,
                    int64_t coef_stride, uint64_t *__restrict__ klo, uint64_t *__restrict__ khi,
                    uint32_t *__restrict__ tag, uint32_t *__restrict__ seen1, uint32_t *__restrict__ seen2,
                    uint64_t seen_mask, int64_t g0, const uint8_t *__restrict__ kst, int kst_stride,
                    const int32_t *__restrict__ single_of, int32_t *__restrict__ ms) {
    const int t = blockIdx.y;
    const int64_t so = (int64_t)t * nsets, nm = nsets - g0;
    uint64_t a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (k < Ks) {
            a[k] = A[t * Ks + k];
            b[k] = B[t * Ks + k];
        }
    int ks = ms ? (int)kst[t] : -1;  // injective function of the instance in a / b
    int have = count > 1 ? -1 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * SM_U;
    for (int64_t gb = g0 + (int64_t)blockIdx.x * blockDim.x * SM_U; gb < nsets; gb += stride) {
        int64_t s0[SM_U], s1[SM_U];
        uint32_t inst[SM_U], m0[SM_U], m1[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; u++) {
            const int64_t g = gb + u * blockDim.x + threadIdx.x;
            const bool in = g < nsets;
            s0[u] = in ? soff[g] : 0;
            s1[u] = in ? soff[g + 1] : 0;
            inst[u] = (in && count > 1) ? set_inst[g] : 0u;
        }
#pragma unroll
        for (int u = 0; u < SM_U; u++) {
            m0[u] = s1[u] > s0[u] ? sids[s0[u]] : 0u;
            m1[u] = s1[u] > s0[u] + 1 ? sids[s0[u] + 1] : 0u;
        }
        uint32_t wpos[SM_U], bit[SM_U];
        int64_t cand[SM_U];  // global id of the matching one-object bucket's object, or -1
#pragma unroll
        for (int u = 0; u < SM_U; u++) {
            const int64_t g = gb + u * blockDim.x + threadIdx.x;
            wpos[u] = 0;
            bit[u] = 0;
            cand[u] = -1;
            if (g >= nsets) continue;
            uint32_t base = 0;
            if (count > 1 && s1[u] > s0[u]) {
                if ((int)inst[u] != have) {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (k < Ks) {
                            a[k] = A[(int64_t)inst[u] * coef_stride + t * Ks + k];
                            b[k] = B[(int64_t)inst[u] * coef_stride + t * Ks + k];
                        }
                    if (ms) ks = (int)kst[(int64_t)inst[u] * kst_stride + t];
                    have = (int)inst[u];
                }
                base = (uint32_t)row_off[inst[u]];
            }
            uint32_t m[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            uint32_t hs = 0xFFFFFFFFu, as = 0;  // injective function: minimum and argmin
            for (int64_t p = s0[u]; p < s1[u]; p++) {
                const uint32_t id = (p == s0[u] ? m0[u] : p == s0[u] + 1 ? m1[u] : sids[p]) - base;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (k < Ks) {
                        const uint32_t h = mh_hash32(a[k], b[k], id);
                        if (k == ks && h < hs) {
                            hs = h;
                            as = id;
                        }
                        m[k] = min(m[k], h);
                    }
            }
            uint64_t hi = 0, lo = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (k < Ks) {
                    hi = (hi << 32) | (lo >> 32);
                    lo = (lo << 32) | m[k];
                }
            const uint32_t tg = count > 1 && s1[u] > s0[u] ? inst[u] : 0u;
            klo[so + g] = lo;
            if (khi) khi[so + g] = hi;
            if (tag) tag[so + g] = tg;
            const uint64_t pos = seen_pos(sig_hash(lo, hi, tg), t, seen_mask);
            wpos[u] = (uint32_t)(pos >> 5);
            bit[u] = 1u << (pos & 31);
            if (ms && s1[u] > s0[u] && ks >= 0 && ks < Ks) {
                bool all = true;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (k < Ks) all = all && mh_hash32(a[k], b[k], as) == m[k];
                if (all) cand[u] = (int64_t)as + base;
            }
        }
        int32_t gi[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; u++) gi[u] = cand[u] >= 0 ? single_of[cand[u]] : -1;
        uint32_t old[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; u++) old[u] = bit[u] ? atomicOr(&seen1[wpos[u]], bit[u]) : 0u;
#pragma unroll
        for (int u = 0; u < SM_U; u++) {
            const int64_t g = gb + u * blockDim.x + threadIdx.x;
            if ((old[u] & bit[u]) || gi[u] >= 0) atomicOr(&seen2[wpos[u]], bit[u]);
            if (ms && g < nsets) ms[t * nm + (g - g0)] = gi[u];
        }
    }
}

// The same signatures for sets of many members: a thread takes one set for
// all S tables (its first SS_REG member ids stay in registers, the per-set
// lookups are paid once), where k_set_sig spends a thread per (set, table).
// With a few members per set the thread per (set, table) keeps more loads in
// flight and is the faster form; with hundreds this one is.
constexpr int SS_REG = 8;
constexpr int64_t SS_WIDE = 32;  // members per set (mean) from which k_set_sig_sets is used
__global__ void k_set_sig_sets(int64_t nsets, int S, const int64_t *__restrict__ soff,
                          const uint32_t *__restrict__ sids, int Ks, const uint64_t *__restrict__ A,
                          const uint64_t *__restrict__ B, const int64_t *__restrict__ row_off, int count,
                          const uint32_t *__restrict__ set_inst, int64_t coef_stride, uint64_t *__restrict__ klo,
                          uint64_t *__restrict__ khi, uint32_t *__restrict__ vals, uint32_t *__restrict__ tag,
                          uint32_t *__restrict__ seen1 = nullptr, uint32_t *__restrict__ seen2 = nullptr,
                          uint64_t seen_mask = 0, int64_t g0 = 0) {
    for (int64_t g = g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nsets;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s0 = soff[g], s1 = soff[g + 1];
        int inst = 0;
        uint32_t base = 0;
        if (count > 1 && s1 > s0) {
            inst = set_inst ? (int)set_inst[g] : find_inst(row_off, count, (int64_t)sids[s0]);
            base = (uint32_t)row_off[inst];
        }
        const uint64_t *Ai = A + (count > 1 ? (int64_t)inst * coef_stride : 0);
        const uint64_t *Bi = B + (count > 1 ? (int64_t)inst * coef_stride : 0);
        const int64_t len = s1 - s0;
        uint32_t mc[SS_REG];
#pragma unroll
        for (int i = 0; i < SS_REG; i++) mc[i] = i < len ? sids[s0 + i] - base : 0u;
        for (int t = 0; t < S; t++) {
            uint64_t a[4], b[4];
            uint32_t m[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (k < Ks) {
                    a[k] = __ldg(Ai + t * Ks + k);
                    b[k] = __ldg(Bi + t * Ks + k);
                }
#pragma unroll
            for (int i = 0; i < SS_REG; i++)
                if (i < len) {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (k < Ks) m[k] = min(m[k], mh_hash32(a[k], b[k], mc[i]));
                }
            for (int64_t p = s0 + SS_REG; p < s1; p++) {
                const uint32_t id = sids[p] - base;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (k < Ks) m[k] = min(m[k], mh_hash32(a[k], b[k], id));
            }
            uint64_t hi = 0, lo = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (k < Ks) {
                    hi = (hi << 32) | (lo >> 32);
                    lo = (lo << 32) | m[k];
                }
            const int64_t so = (int64_t)t * nsets;
            klo[so + g] = lo;
            if (khi) khi[so + g] = hi;
            if (vals) vals[so + g] = (uint32_t)g;
            if (tag) tag[so + g] = (uint32_t)inst;
            if (seen1) {
                const uint64_t pos = seen_pos(sig_hash(lo, hi, (uint32_t)inst), t, seen_mask);
                const uint32_t bit = 1u << (pos & 31);
                if (atomicOr(&seen1[pos >> 5], bit) & bit) atomicOr(&seen2[pos >> 5], bit);
            }
        }
    }
}

// first signature component (the most significant 32 bits of the packed
// key), with the instance tag (if any) above it
__global__ void k_first_component(int64_t n, const uint64_t *__restrict__ klo, const uint64_t *__restrict__ khi,
                                  const uint32_t *__restrict__ tag, int Ks, uint64_t *__restrict__ k0) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        uint64_t v;
        if (Ks == 1) v = klo[g];
        else if (Ks == 2) v = klo[g] >> 32;
        else if (Ks == 3) v = khi[g];
        else v = khi[g] >> 32;
        k0[g] = (v & 0xFFFFFFFFull) | (tag ? (uint64_t)tag[g] << 32 : 0ull);
    }
}

__device__ __forceinline__ bool sig_less(const uint64_t *klo, const uint64_t *khi, uint32_t a, uint32_t b) {
    const uint64_t ha = khi ? khi[a] : 0, hb = khi ? khi[b] : 0;
    if (ha != hb) return ha < hb;
    if (klo[a] != klo[b]) return klo[a] < klo[b];
    return a < b;
}

// insertion sort of each run of equal first components by (signature, index);
// blockIdx.y = segment
__global__ void k_fix_runs(int64_t m, const int64_t *__restrict__ runs, const int64_t *__restrict__ rs_all,
                           const uint64_t *__restrict__ klo_all, const uint64_t *__restrict__ khi_all,
                           uint32_t *__restrict__ perm_all) {
    const int t = blockIdx.y;
    const int64_t *rs = rs_all + (int64_t)t * (m + 1);
    const uint64_t *klo = klo_all + (int64_t)t * m;
    const uint64_t *khi = khi_all ? khi_all + (int64_t)t * m : nullptr;
    uint32_t *perm = perm_all + (int64_t)t * m;
    const int64_t nr = runs[t];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = rs[r], e = rs[r + 1];
        for (int64_t i = s + 1; i < e; i++) {
            const uint32_t v = perm[i];
            int64_t j = i - 1;
            while (j >= s && sig_less(klo, khi, v, perm[j])) {
                perm[j + 1] = perm[j];
                j--;
            }
            perm[j + 1] = v;
        }
    }
}

__global__ void k_gather_sig(int64_t m, int S, const uint32_t *__restrict__ perm, const uint64_t *__restrict__ klo,
                             const uint64_t *__restrict__ khi, const uint32_t *__restrict__ tag,
                             uint64_t *__restrict__ slo, uint64_t *__restrict__ shi, uint32_t *__restrict__ stag) {
    const int64_t tot = m * S;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < tot; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t so = (p / m) * m;
        const uint32_t g = perm[p];
        slo[p] = klo[so + g];
        if (shi) shi[p] = khi[so + g];
        if (stag) stag[p] = tag[so + g];
    }
}

// per-segment bin numbering -> one global numbering over all segments
__global__ void k_globalize_rank(int64_t m, int S, const int64_t *__restrict__ base, int32_t *__restrict__ rank) {
    const int64_t tot = m * S;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < tot; p += (int64_t)gridDim.x * blockDim.x)
        rank[p] += (int32_t)base[p / m];
}

__global__ void k_globalize_rs(int64_t m, const int64_t *__restrict__ runs, const int64_t *__restrict__ base,
                               const int64_t *__restrict__ rs_seg, int64_t *__restrict__ rs_g, int S) {
    const int t = blockIdx.y;
    const int64_t nr = runs[t];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x)
        rs_g[base[t] + r] = (int64_t)t * m + rs_seg[(int64_t)t * (m + 1) + r];
    if (t == S - 1 && blockIdx.x == 0 && threadIdx.x == 0) rs_g[base[t] + nr] = (int64_t)S * m;
}

__device__ __forceinline__ int64_t bin_size(const int64_t *rs, int64_t r) { return rs[r + 1] - rs[r]; }

// member count of each sorted position whose bin qualifies for a vote
__global__ void k_vote_weights(int64_t m, const int32_t *__restrict__ rank,
                               const int64_t *__restrict__ rs, const uint32_t *__restrict__ perm,
                               const int64_t *__restrict__ soff, int64_t *__restrict__ w) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rank[p];
        const uint32_t g = perm[p];
        w[p] = bin_size(rs, r) >= 2 ? soff[g + 1] - soff[g] : 0;
    }
}

__global__ void k_vote_expand(int64_t m, const int32_t *__restrict__ rank,
                              const uint32_t *__restrict__ perm, const int64_t *__restrict__ woff,
                              const int64_t *__restrict__ w, const int64_t *__restrict__ soff,
                              const uint32_t *__restrict__ sids, uint64_t *__restrict__ pairs) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (w[p] == 0) continue;
        const uint64_t r = (uint64_t)rank[p];
        const uint32_t g = perm[p];
        int64_t o = woff[p];
        for (int64_t q = soff[g]; q < soff[g + 1]; q++) pairs[o++] = (r << 32) | sids[q];
    }
}

// one thread per (bin, id) run: keep when 2 * count > |bin|
__global__ void k_vote_keep(const int64_t *__restrict__ nruns_dev, const int64_t *__restrict__ prs,
                            const uint64_t *__restrict__ pairs, const int64_t *__restrict__ rs,
                            int64_t *__restrict__ keep, int64_t *__restrict__ cnt) {
    const int64_t nr = *nruns_dev;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = prs[r + 1] - prs[r];
        const int64_t bin = (int64_t)(pairs[prs[r]] >> 32);
        const bool k = 2 * len > bin_size(rs, bin);
        keep[r] = k;
        if (k) atomicAdd((unsigned long long *)&cnt[bin], 1ull);
    }
}

// per bin: ok when it has >= 2 buckets and |C_shared| >= delta
__global__ void k_bin_ok(int64_t nbins, const int64_t *__restrict__ rs, const int64_t *__restrict__ cnt,
                         int delta, int64_t *__restrict__ ok, int64_t *__restrict__ len) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x) {
        const bool o = bin_size(rs, b) >= 2 && cnt[b] >= delta;
        ok[b] = o;
        len[b] = o ? cnt[b] : 0;
    }
}

__global__ void k_vote_sel(const int64_t *__restrict__ nruns_dev, const int64_t *__restrict__ prs,
                           const uint64_t *__restrict__ pairs, const int64_t *__restrict__ keep,
                           const int64_t *__restrict__ ok, int64_t *__restrict__ sel) {
    const int64_t nr = *nruns_dev;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bin = (int64_t)(pairs[prs[r]] >> 32);
        sel[r] = keep[r] && ok[bin];
    }
}

__global__ void k_vote_emit(const int64_t *__restrict__ nruns_dev, const int64_t *__restrict__ prs,
                            const uint64_t *__restrict__ pairs, const int64_t *__restrict__ sel,
                            const int64_t *__restrict__ pos, uint32_t *__restrict__ out_ids) {
    const int64_t nr = *nruns_dev;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x)
        if (sel[r]) out_ids[pos[r]] = (uint32_t)(pairs[prs[r]] & 0xFFFFFFFFu);
}

__global__ void k_compact_offsets(int64_t nbins, const int64_t *__restrict__ ok,
                                  const int64_t *__restrict__ set_idx, const int64_t *__restrict__ boffs,
                                  int64_t *__restrict__ out_off, const int64_t *__restrict__ nsets,
                                  const int64_t *__restrict__ total) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x)
        if (ok[b]) out_off[set_idx[b]] = boffs[b];
    if (blockIdx.x == 0 && threadIdx.x == 0) out_off[*nsets] = *total;
}

// set lengths of a list of set indices
__global__ void k_gather_len(int64_t cnt, const int64_t *__restrict__ idx, const int64_t *__restrict__ soff,
                             int64_t *__restrict__ len) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        len[i] = soff[idx[i] + 1] - soff[idx[i]];
}

__global__ void k_gather_ids(int64_t cnt, const int64_t *__restrict__ idx, const int64_t *__restrict__ soff,
                             const uint32_t *__restrict__ sids, const int64_t *__restrict__ ooff,
                             uint32_t *__restrict__ oids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx[i];
        int64_t o = ooff[i];
        for (int64_t q = soff[s]; q < soff[s + 1]; q++) oids[o++] = sids[q];
    }
}

__device__ int set_cmp(const uint32_t *ids, const int64_t *off, int64_t a, int64_t b) {
    const int64_t na = off[a + 1] - off[a], nb = off[b + 1] - off[b];
    const int64_t m = na < nb ? na : nb;
    const uint32_t *pa = ids + off[a], *pb = ids + off[b];
    for (int64_t i = 0; i < m; i++)
        if (pa[i] != pb[i]) return pa[i] < pb[i] ? -1 : 1;
    return (na > nb) - (na < nb);
}

// dedup bins: classify each bin of sets.  Singleton bins contribute their
// set (kind 1); bins with >= 2 sets whose vote failed delta contribute their
// canonically smallest member (kind 2).
__global__ void k_dedup_pick(int64_t nbins, const int64_t *__restrict__ rs, const uint32_t *__restrict__ perm,
                             const int64_t *__restrict__ ok, const int64_t *__restrict__ soff,
                             const uint32_t *__restrict__ sids, int64_t *__restrict__ pick,
                             int64_t *__restrict__ has) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = rs[b], e = rs[b + 1];
        if (e - s == 1) {
            pick[b] = perm[s];
            has[b] = 1;
        } else if (!ok[b]) {
            int64_t best = perm[s];
            for (int64_t p = s + 1; p < e; p++)
                if (set_cmp(sids, soff, perm[p], best) < 0) best = perm[p];
            pick[b] = best;
            has[b] = 1;
        } else {
            has[b] = 0;
        }
    }
}

__global__ void k_compact_idx(int64_t nb, const int64_t *__restrict__ has, const int64_t *__restrict__ pos,
                              const int64_t *__restrict__ val, int64_t *__restrict__ out) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (int64_t)gridDim.x * blockDim.x)
        if (has[b]) out[pos[b]] = val[b];
}

// canonical order: 64-bit prefix key (first two members + 1, 0 if absent)
__global__ void k_prefix_key(int64_t ns, const int64_t *__restrict__ soff, const uint32_t *__restrict__ sids,
                             uint64_t *__restrict__ key, uint32_t *__restrict__ vals) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = soff[s + 1] - soff[s];
        const uint64_t a = n > 0 ? (uint64_t)sids[soff[s]] + 1 : 0;
        const uint64_t b = n > 1 ? (uint64_t)sids[soff[s] + 1] + 1 : 0;
        key[s] = (a << 32) | b;
        vals[s] = (uint32_t)s;
    }
}

// within each run of equal prefix keys, order by full comparison (ties by
// position, so the order is total): final[run_start + rank] = set
__global__ void k_prefix_fix(int64_t ns, const int32_t *__restrict__ rank, const int64_t *__restrict__ rs,
                             const uint32_t *__restrict__ perm, const int64_t *__restrict__ soff,
                             const uint32_t *__restrict__ sids, int64_t *__restrict__ order) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ns;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rank[p], s = rs[r], e = rs[r + 1];
        int64_t c = 0;
        for (int64_t q = s; q < e; q++) {
            if (q == p) continue;
            const int cmp = set_cmp(sids, soff, perm[q], perm[p]);
            if (cmp < 0 || (cmp == 0 && q < p)) c++;
        }
        order[s + c] = perm[p];
    }
}

__global__ void k_dup_flags(int64_t ns, const int64_t *__restrict__ order, const int64_t *__restrict__ soff,
                            const uint32_t *__restrict__ sids, int64_t *__restrict__ keep) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ns;
         p += (int64_t)gridDim.x * blockDim.x)
        keep[p] = p == 0 || set_cmp(sids, soff, order[p - 1], order[p]) != 0;
}

// ---- virtual buckets ---------------------------------------------------------
// Identical buckets always share a bin and contribute identically to its
// vote, so the main pass works on distinct "virtual buckets" with a
// multiplicity: every object whose bucket is a singleton in m >= 1 tables
// gives one virtual bucket {i} of weight m; every bucket of two or more
// objects is its own virtual bucket of weight 1.  A bin's size |Bin| is the
// total weight of its virtual buckets and an object's count the total weight
// of those containing it, exactly as in Alg. 4 over the original buckets.
__global__ void k_vb_count(int64_t NB, const int64_t *__restrict__ boff, const uint32_t *__restrict__ mem,
                           int32_t *__restrict__ mult, int64_t *__restrict__ ns_flag) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < NB; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sz = boff[g + 1] - boff[g];
        if (sz == 1) atomicAdd(&mult[mem[boff[g]]], 1);
        ns_flag[g] = sz >= 2;
    }
}

__global__ void k_pos_flag(int64_t n, const int32_t *__restrict__ mult, int64_t *__restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = mult[i] > 0;
}

// (single_of[i]: the one-object virtual bucket {i}, or -1)
__global__ void k_vb_fill_s(int64_t n, const int32_t *__restrict__ mult, const int64_t *__restrict__ pos,
                            int64_t *__restrict__ vsz, int32_t *__restrict__ vw, int64_t *__restrict__ vsrc,
                            int32_t *__restrict__ single_of) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        single_of[i] = mult[i] > 0 ? (int32_t)pos[i] : -1;
        if (mult[i] > 0) {
            const int64_t v = pos[i];
            vsz[v] = 1;
            vw[v] = mult[i];
            vsrc[v] = i;
        }
    }
}

__global__ void k_vb_fill_n(int64_t NB, const int64_t *__restrict__ boff, const int64_t *__restrict__ ns_flag,
                            const int64_t *__restrict__ pos, int64_t base, int64_t *__restrict__ vsz,
                            int32_t *__restrict__ vw, int64_t *__restrict__ vsrc) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < NB; g += (int64_t)gridDim.x * blockDim.x)
        if (ns_flag[g]) {
            const int64_t v = base + pos[g];
            vsz[v] = boff[g + 1] - boff[g];
            vw[v] = 1;
            vsrc[v] = g;
        }
}

__global__ void k_vb_members(int64_t NV, int64_t NS1, const int64_t *__restrict__ vsrc,
                             const int64_t *__restrict__ voff, const int64_t *__restrict__ boff,
                             const uint32_t *__restrict__ mem, uint32_t *__restrict__ vmem) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < NV; v += (int64_t)gridDim.x * blockDim.x) {
        if (v < NS1) {
            vmem[voff[v]] = (uint32_t)vsrc[v];
        } else {
            const int64_t g = vsrc[v];
            int64_t o = voff[v];
            for (int64_t q = boff[g]; q < boff[g + 1]; q++) vmem[o++] = mem[q];
        }
    }
}

// per bin: number of virtual buckets and total weight |Bin|
__global__ void k_bin_weight(int64_t nbins, const int64_t *__restrict__ rs, const uint32_t *__restrict__ perm,
                             const int32_t *__restrict__ vw, int64_t *__restrict__ bw) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nbins; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int64_t p = rs[r]; p < rs[r + 1]; p++) s += vw[perm[p]];
        bw[r] = s;
    }
}

// weighted vote over bins of >= 2 virtual buckets
// A bin in which one single-object virtual bucket {a} holds at least half
// of the weight |Bin| keeps at most a: any other object is counted at most
// |Bin| - m_a <= |Bin| / 2 times.  With delta >= 2 such a bin yields nothing
// and skips the vote (pruned[bin] = 1).
__global__ void k_bin_prune(int64_t nbins, const int64_t *__restrict__ rs, const uint32_t *__restrict__ perm,
                            const int32_t *__restrict__ vw, const int64_t *__restrict__ voff,
                            const int64_t *__restrict__ bw, int delta, uint8_t *__restrict__ pruned) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nbins; r += (int64_t)gridDim.x * blockDim.x) {
        bool pr = false;
        if (delta >= 2)
            for (int64_t q = rs[r]; q < rs[r + 1] && !pr; q++) {
                const uint32_t v = perm[q];
                pr = voff[v + 1] - voff[v] == 1 && 2 * (int64_t)vw[v] >= bw[r];
            }
        pruned[r] = pr;
    }
}

__global__ void k_wvote_weights(int64_t m, const int32_t *__restrict__ rank, const int64_t *__restrict__ rs,
                                const uint32_t *__restrict__ perm, const int64_t *__restrict__ voff,
                                const uint8_t *__restrict__ pruned, int64_t *__restrict__ w) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rank[p];
        const uint32_t v = perm[p];
        w[p] = (bin_size(rs, r) >= 2 && !(pruned && pruned[r])) ? voff[v + 1] - voff[v] : 0;
    }
}

__global__ void k_wvote_expand(int64_t m, const int32_t *__restrict__ rank, const uint32_t *__restrict__ perm,
                               const int64_t *__restrict__ woff, const int64_t *__restrict__ w,
                               const int64_t *__restrict__ voff, const uint32_t *__restrict__ vmem,
                               const int32_t *__restrict__ vw, uint64_t *__restrict__ pairs,
                               uint32_t *__restrict__ pw) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (w[p] == 0) continue;
        const uint64_t r = (uint64_t)rank[p];
        const uint32_t v = perm[p];
        int64_t o = woff[p];
        for (int64_t q = voff[v]; q < voff[v + 1]; q++) {
            pw[o] = (uint32_t)vw[v];
            pairs[o++] = (r << 32) | vmem[q];
        }
    }
}

__global__ void k_wvote_keep(const int64_t *__restrict__ nruns_dev, const int64_t *__restrict__ prs,
                             const uint64_t *__restrict__ pairs, const uint32_t *__restrict__ pw,
                             const int64_t *__restrict__ bw, int64_t *__restrict__ keep, int64_t *__restrict__ cnt) {
    const int64_t nr = *nruns_dev;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int64_t q = prs[r]; q < prs[r + 1]; q++) c += pw[q];
        const int64_t bin = (int64_t)(pairs[prs[r]] >> 32);
        const bool k = 2 * c > bw[bin];
        keep[r] = k;
        if (k) atomicAdd((unsigned long long *)&cnt[bin], 1ull);
    }
}

__global__ void k_wbin_ok(int64_t nbins, const int64_t *__restrict__ rs, const int64_t *__restrict__ cnt, int delta,
                          int64_t *__restrict__ ok, int64_t *__restrict__ len) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const bool o = bin_size(rs, b) >= 2 && cnt[b] >= delta;
        ok[b] = o;
        len[b] = o ? cnt[b] : 0;
    }
}

// ---- exact grouping of equal signatures by hashing ---------------------------
// Segment t (a SILK table) has a table of C slots (C a power of two >= 2 NV,
// so probing always ends).  A slot holds, in its low 31 bits, the index g of
// the first set that claimed it; sets whose full signature (and instance tag)
// equals that set's join its group, and the first joiner sets bit 31 (the
// group has >= 2 sets).  grp[p] = the slot of position p's group.
// A slot is 64 bits: a 32-bit fingerprint of the signature (high word) and
// the group's first set g | SLOT_MULTI (low word; g < 2^31 - 1, so a used
// slot never equals SLOT_EMPTY).  Probes compare fingerprints first and read
// the first set's signature only on a fingerprint match.
constexpr uint64_t SLOT_EMPTY = ~0ull;
constexpr uint32_t SLOT_MULTI = 0x80000000u;

// Block-aggregated append (256 threads, block-uniform call): one atomic per
// block and list, so that a list filled by every block does not serialise
// on one counter.  Thread t appends c entries (c >= 0); returns the first of
// its positions.
constexpr int AP_THREADS = 256;
__device__ __forceinline__ unsigned long long block_append_n(unsigned c, unsigned long long *counter,
                                                             unsigned *wcnt /* [AP_THREADS / 32] shared */,
                                                             unsigned long long *base /* shared */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = c;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wcnt[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int w = 0; w < AP_THREADS / 32; w++) {
            const unsigned v = wcnt[w];
            wcnt[w] = run;
            run += v;
        }
        *base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    const unsigned long long q = *base + wcnt[warp] + (x - c);
    __syncthreads();  // wcnt / base reused by the next call
    return q;
}
__device__ __forceinline__ unsigned long long block_append(bool want, unsigned long long *counter, unsigned *wcnt,
                                                           unsigned long long *base) {
    return block_append_n(want ? 1u : 0u, counter, wcnt, base);
}

// Batched instances: instance i owns the slot region [roff[i], roff[i] +
// rcap[i]) (rcap a power of two >= 2x its sets), so a block, whose sets mostly
// belong to one instance, probes one small region.  A set that joins an
// existing group appends itself to the multi list (key = segment * C + slot);
// the one joiner that sets the group's SLOT_MULTI bit also appends the
// group's first set, so every group of >= 2 sets is listed whole.
// With ms given (k_set_sig_marks), a set whose signature equals that of the
// one-object bucket ms[...] claims it in the claimed map (one bit per table
// and one-object bucket): the one claimant appends the bucket to its group,
// which then holds >= 2 sets, with the group's first set as above.
//
// A thread takes GI_U sets at a time: their signature loads, seen-twice
// reads and first slot reads are in flight together.
constexpr int GI_U = 4;
__global__ void __launch_bounds__(AP_THREADS, 3)
    k_group_insert(int64_t NV, int64_t C, const uint64_t *__restrict__ klo, const uint64_t *__restrict__ khi,
                   const uint32_t *__restrict__ tag, const int64_t *__restrict__ roff,
                   const int64_t *__restrict__ rcap, uint64_t *__restrict__ slot, uint64_t *__restrict__ mkey,
                   uint32_t *__restrict__ mval, unsigned long long *__restrict__ n_multi,
                   const uint32_t *__restrict__ seen2, uint64_t seen_mask, const int32_t *__restrict__ vw,
                   const int64_t *__restrict__ voff, int delta, int64_t *__restrict__ singles,
                   unsigned long long *__restrict__ n_single, int64_t g0, const int32_t *__restrict__ ms,
                   uint32_t *__restrict__ claimed, int64_t claimed_words) {
    // sets g0 .. NV-1 of segment t = blockIdx.y (NV is the segment stride)
    const int t = blockIdx.y;
    const int64_t so = (int64_t)t * NV, nm = NV - g0;
    uint64_t *sl = slot + (int64_t)t * C;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * GI_U;
    __shared__ unsigned s_wc[AP_THREADS / 32];
    __shared__ unsigned long long s_base;
    // the whole block iterates together (the append is a block collective)
    for (int64_t gb = g0 + (int64_t)blockIdx.x * blockDim.x * GI_U; gb < NV; gb += stride) {
        uint64_t lo[GI_U], hi[GI_U], hf[GI_U];
        uint32_t tg[GI_U];
        int32_t gi[GI_U];
#pragma unroll
        for (int u = 0; u < GI_U; u++) {
            const int64_t g = gb + u * blockDim.x + threadIdx.x;
            const bool in = g < NV;
            lo[u] = in ? klo[so + g] : 0;
            hi[u] = (in && khi) ? khi[so + g] : 0;
            tg[u] = (in && tag) ? tag[so + g] : 0;
            gi[u] = (in && ms) ? ms[t * nm + (g - g0)] : -1;
        }
        unsigned go = 0;  // bit u: set u probes the grouping table
        uint32_t bits[GI_U];
#pragma unroll
        for (int u = 0; u < GI_U; u++) {
            hf[u] = sig_hash(lo[u], hi[u], tg[u]);
            bits[u] = 0;
            if (gb + u * blockDim.x + threadIdx.x < NV) {
                if (seen2) bits[u] = seen2[seen_pos(hf[u], t, seen_mask) >> 5];
                go |= 1u << u;
            }
        }
        unsigned sm = 0;  // bit u: set u is alone in its bin and a single-bin candidate
#pragma unroll
        for (int u = 0; u < GI_U; u++)
            if (((go >> u) & 1u) && seen2 && !((bits[u] >> (seen_pos(hf[u], t, seen_mask) & 31)) & 1u)) {
                go &= ~(1u << u);  // alone in its bin
                const int64_t g = gb + u * blockDim.x + threadIdx.x;
                if (delta <= 1 && vw[g] >= 2 && voff[g + 1] - voff[g] >= delta) sm |= 1u << u;
            }
        uint64_t cur0[GI_U];
#pragma unroll
        for (int u = 0; u < GI_U; u++) {
            cur0[u] = SLOT_EMPTY;
            if ((go >> u) & 1u) {
                const int64_t base = tag ? roff[tg[u]] : 0;
                const uint64_t mask = (uint64_t)(tag ? rcap[tg[u]] : C) - 1;
                cur0[u] = sl[base + (hf[u] & mask)];
            }
        }
        unsigned jm = 0, fm = 0, cm = 0;  // joined / appends the group's first set / claimed gi
        uint64_t key[GI_U];
        uint32_t rep[GI_U];
#pragma unroll
        for (int u = 0; u < GI_U; u++) {
            key[u] = 0;
            rep[u] = 0;
            if (!((go >> u) & 1u)) continue;
            const int64_t g = gb + u * blockDim.x + threadIdx.x;
            const int64_t base = tag ? roff[tg[u]] : 0;
            const uint64_t mask = (uint64_t)(tag ? rcap[tg[u]] : C) - 1;
            const uint32_t fp = (uint32_t)(hf[u] >> 32);
            const uint64_t mine = ((uint64_t)fp << 32) | (uint64_t)g;
            uint64_t h = hf[u] & mask;
            uint64_t cur = cur0[u];
            for (uint64_t probe = 0; probe <= mask; probe++) {
                unsigned long long *ps = (unsigned long long *)&sl[base + h];
                if (probe) cur = *ps;
                if (cur == SLOT_EMPTY) {
                    const uint64_t prev = atomicCAS(ps, (unsigned long long)SLOT_EMPTY, (unsigned long long)mine);
                    if (prev == SLOT_EMPTY) {  // first set of a new group
                        rep[u] = (uint32_t)g;
                        key[u] = (uint64_t)t * (uint64_t)C + (uint64_t)(base + h);
                        break;
                    }
                    cur = prev;
                }
                if ((uint32_t)(cur >> 32) == fp) {
                    const uint32_t r = (uint32_t)cur & ~SLOT_MULTI;
                    const uint64_t rlo = klo[so + r], rhi = khi ? khi[so + r] : 0;
                    const uint32_t rtg = tag ? tag[so + r] : 0;
                    if (rlo == lo[u] && rhi == hi[u] && rtg == tg[u]) {
                        if (!(cur & SLOT_MULTI) && !(atomicOr(ps, (unsigned long long)SLOT_MULTI) & SLOT_MULTI))
                            fm |= 1u << u;
                        rep[u] = r;
                        jm |= 1u << u;
                        key[u] = (uint64_t)t * (uint64_t)C + (uint64_t)(base + h);
                        break;
                    }
                }
                h = (h + 1) & mask;
            }
            if (gi[u] >= 0) {  // claim the one-object bucket with this signature
                const uint32_t cb = 1u << (gi[u] & 31);
                if (!(atomicOr(&claimed[t * claimed_words + (gi[u] >> 5)], cb) & cb)) {
                    cm |= 1u << u;
                    if (!(atomicOr((unsigned long long *)&slot[key[u]], (unsigned long long)SLOT_MULTI) & SLOT_MULTI))
                        fm |= 1u << u;
                }
            }
        }
        const unsigned long long q =
            block_append_n(__popc(jm) + __popc(fm) + __popc(cm), n_multi, s_wc, &s_base);
        int w = 0;
#pragma unroll
        for (int u = 0; u < GI_U; u++) {
            if ((jm >> u) & 1u) {
                mkey[q + w] = key[u];
                mval[q + w] = (uint32_t)(gb + u * blockDim.x + threadIdx.x);
                w++;
            }
            if ((fm >> u) & 1u) {
                mkey[q + w] = key[u];
                mval[q + w] = rep[u];
                w++;
            }
            if ((cm >> u) & 1u) {
                mkey[q + w] = key[u];
                mval[q + w] = (uint32_t)gi[u];
                w++;
            }
        }
        if (delta <= 1 && __syncthreads_or(sm)) {  // (block-uniform)
            const unsigned long long qs = block_append_n(__popc(sm), n_single, s_wc, &s_base);
            int ws = 0;
#pragma unroll
            for (int u = 0; u < GI_U; u++)
                if ((sm >> u) & 1u) singles[qs + ws++] = gb + u * blockDim.x + threadIdx.x;
        }
    }
}

// delta <= 1 with one-object buckets claimed (k_group_insert): a one-object
// bucket that no set of table t claimed is alone in its bin, and with weight
// >= 2 that bin keeps it (one object >= delta).
__global__ void k_single_unclaimed(int64_t ns1, const uint32_t *__restrict__ claimed, int64_t claimed_words,
                                   const int32_t *__restrict__ vw, int64_t *__restrict__ singles,
                                   unsigned long long *__restrict__ n_single) {
    const int t = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    __shared__ unsigned s_wc[AP_THREADS / 32];
    __shared__ unsigned long long s_base;
    for (int64_t gb = (int64_t)blockIdx.x * blockDim.x; gb < ns1; gb += stride) {
        const int64_t g = gb + threadIdx.x;
        const bool single =
            g < ns1 && vw[g] >= 2 && !((claimed[t * claimed_words + (g >> 5)] >> (g & 31)) & 1u);
        if (__syncthreads_or(single)) {  // (block-uniform)
            const unsigned long long qs = block_append(single, n_single, s_wc, &s_base);
            if (single) singles[qs] = g;
        }
    }
}

// MinHash function h(x) = floor(((A x + B) mod 2^64) / 2^32) (Eq. 2's
// permutation) can take one value at ids x and x + q only if the two 64-bit
// values share their high word, which needs A q mod 2^64 within 2^32 of a
// multiple of 2^64.  So h is injective on ids [0, n) when no q in [1, n) has
// that property; a thread takes one q (global row r, q = r - the first row of
// its instance) and tests every function (t, k) of the instance, setting
// bit k of fb[instance * Ls + t] when one may repeat a value.
__global__ void k_mh_injective(int64_t N, const int64_t *__restrict__ row_off, int count,
                               const uint64_t *__restrict__ A, int64_t coef_stride, int Ls, int Ks,
                               uint32_t *__restrict__ fb) {
    const int nf = Ls * Ks;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
        const int inst = count > 1 ? find_inst(row_off, count, r) : 0;
        const uint64_t q = (uint64_t)(r - (count > 1 ? row_off[inst] : 0));
        if (q == 0) continue;
        const uint64_t *Ai = A + (int64_t)inst * coef_stride;
        for (int f = 0; f < nf; f++) {
            const uint64_t p = Ai[f] * q;
            const uint32_t ph = (uint32_t)(p >> 32);
            if (ph == 0u || (ph == 0xFFFFFFFFu && (uint32_t)p != 0u))
                atomicOr(&fb[inst * Ls + f / Ks], 1u << (f % Ks));
        }
    }
}

// With delta <= 1, one pass over the slots: a set alone in its group with
// weight >= 2 is a bin of one virtual bucket that keeps the whole bucket
// (with delta >= 2 that rule cannot fire: weight >= 2 only for one-object
// buckets, and the pass is skipped).
__global__ void k_group_singles(int64_t C, int S, const uint64_t *__restrict__ slot, const int32_t *__restrict__ vw,
                                const int64_t *__restrict__ voff, int delta, int64_t *__restrict__ singles,
                                unsigned long long *__restrict__ n_single) {
    const int64_t tot = C * S;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    __shared__ unsigned s_wc[AP_THREADS / 32];
    __shared__ unsigned long long s_base;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < tot; b += stride) {
        const int64_t e = b + threadIdx.x;
        const uint64_t v = e < tot ? slot[e] : SLOT_EMPTY;
        const bool used = v != SLOT_EMPTY;
        const bool multi = used && ((uint32_t)v & SLOT_MULTI);
        const uint32_t g = (uint32_t)v & ~SLOT_MULTI;
        const bool single = used && !multi && vw[g] >= 2 && voff[g + 1] - voff[g] >= delta;
        if (__syncthreads_or(single)) {  // (block-uniform: single-bin sets are rare)
            const unsigned long long qs = block_append(single, n_single, s_wc, &s_base);
            if (single) singles[qs] = g;
        }
    }
}

// sets per instance (the instance of a set is that of its first member);
// lanes of a warp with the same instance add once
// (cnt[count + i]: the sets of instance i from set g_multi on)
__global__ void k_sets_per_inst(int64_t nsets, const int64_t *__restrict__ soff, const uint32_t *__restrict__ sids,
                                const int64_t *__restrict__ row_off, int count, int64_t g_multi,
                                unsigned long long *__restrict__ cnt, uint32_t *__restrict__ set_inst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nsets; base += stride) {
        const int64_t g = base + threadIdx.x;
        const int i = g < nsets ? find_inst(row_off, count, (int64_t)sids[soff[g]]) : -1;
        if (g < nsets) set_inst[g] = (uint32_t)i;
        const unsigned peers = __match_any_sync(0xffffffffu, i);
        if (i >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[i], (unsigned long long)__popc(peers));
        const int im = g >= g_multi ? i : -1;
        const unsigned pm = __match_any_sync(0xffffffffu, im);
        if (im >= 0 && lane == __ffs(pm) - 1) atomicAdd(&cnt[count + im], (unsigned long long)__popc(pm));
    }
}


struct Csr {
    int64_t n = 0;        // sets
    int64_t nids = 0;     // members
    int64_t *off = nullptr;
    uint32_t *ids = nullptr;
};

int G(geek_ctx *ctx, int64_t work) { return grid_for(std::max<int64_t>(work, 1), 256, ctx->num_sms); }

geek_status d2h_i64(geek_ctx *ctx, const int64_t *dev, int64_t *host, cudaStream_t st) {
    GK_CUDA(ctx, cudaMemcpyAsync(host, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    return GEEK_OK;
}

// Group nsets sets into bins by their Ks-function MinHash signature.
// Returns perm (set index per sorted position), rank (bin per position),
// rs (bin starts, nbins + 1) and nbins.
// Groups nsets sets into bins by their Ks-function MinHash signature, for S
// SILK tables at once (segment t uses functions A/B[t*Ks ..]).  Returns, over
// all S*nsets positions: perm (set index), rank (global bin id), rs (global
// bin starts, nbins + 1) and nbins; bins of table t precede those of t + 1.
geek_status make_bins(geek_ctx *ctx, Scratch &scr, int S, int64_t nsets, const int64_t *soff,
                      const uint32_t *sids, int64_t nids, int Ks, const uint64_t *A, const uint64_t *B, const SilkBatch *bt,
                      int64_t coef_stride, uint32_t **perm, int32_t **rank, int64_t **rs, int64_t *nbins,
                      cudaStream_t st) {
    const int64_t tot = (int64_t)S * nsets;
    const bool tagged = bt && bt->count > 1;
    uint64_t *klo, *khi = nullptr, *k0, *slo, *shi = nullptr;
    uint32_t *tag = nullptr, *stag = nullptr;
    GK_TRY(scr.alloc(&klo, tot));
    if (Ks > 2) GK_TRY(scr.alloc(&khi, tot));
    GK_TRY(scr.alloc(&k0, tot));
    GK_TRY(scr.alloc(&slo, tot));
    if (Ks > 2) GK_TRY(scr.alloc(&shi, tot));
    if (tagged) {
        GK_TRY(scr.alloc(&tag, tot));
        GK_TRY(scr.alloc(&stag, tot));
    }
    GK_TRY(scr.alloc(perm, tot));
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nsets, 256), (int64_t)ctx->num_sms * 8));
    GK_COUNT();
    if (nids >= SS_WIDE * nsets)
        k_set_sig_sets<<<gx, 256, 0, st>>>(nsets, S, soff, sids, Ks, A, B, tagged ? bt->row_off : nullptr,
                                           tagged ? bt->count : 1, nullptr, coef_stride, klo, khi, *perm, tag);
    else
        k_set_sig<<<dim3(gx, S), 256, 0, st>>>(nsets, soff, sids, Ks, A, B, tagged ? bt->row_off : nullptr,
                                               tagged ? bt->count : 1, nullptr, coef_stride, klo, khi, *perm, tag);
    GK_COUNT();
    k_first_component<<<G(ctx, tot), 256, 0, st>>>(tot, klo, khi, tag, Ks, k0);
    GK_LAUNCH(ctx);
    // stable sort by (instance, first component), then order every run of
    // equal first components by the whole signature (runs are short: sets
    // sharing a first component share that component's argmin object, which
    // lies in at most one bucket per table, unless 32-bit values collide)
    const int k0bits = 32 + (tagged ? bit_length_u64((uint64_t)(bt->count - 1)) : 0);
    GK_TRY(radix_sort_segments(ctx, scr, S, nsets, &k0, nullptr, perm, k0bits, st));
    int64_t *runs0, *rs0;
    GK_TRY(scr.alloc(&runs0, S));
    GK_TRY(scr.alloc(&rs0, (size_t)S * (nsets + 1)));
    GK_TRY(segment_runs(ctx, scr, S, nsets, k0, nullptr, nullptr, rs0, runs0, st));
    if (Ks > 1) {
        GK_COUNT();
        k_fix_runs<<<dim3(gx, S), 256, 0, st>>>(nsets, runs0, rs0, klo, khi, *perm);
    }
    GK_COUNT();
    k_gather_sig<<<G(ctx, tot), 256, 0, st>>>(nsets, S, *perm, klo, khi, tag, slo, shi, stag);
    GK_LAUNCH(ctx);
    int64_t *runs, *rs_seg, *d_base;
    GK_TRY(scr.alloc(rank, tot));
    GK_TRY(scr.alloc(&rs_seg, (size_t)S * (nsets + 1)));
    GK_TRY(scr.alloc(&runs, S));
    GK_TRY(scr.alloc(&d_base, S));
    GK_TRY(segment_runs_tagged(ctx, scr, S, nsets, slo, shi, stag, *rank, rs_seg, runs, st));
    std::vector<int64_t> h_runs(S), h_base(S);
    GK_CUDA(ctx, cudaMemcpyAsync(h_runs.data(), runs, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t total = 0, maxr = 1;
    for (int t = 0; t < S; t++) {
        h_base[t] = total;
        total += h_runs[t];
        maxr = std::max(maxr, h_runs[t]);
    }
    if (total > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 2^31 SILK bins in one pass");
    GK_CUDA(ctx, cudaMemcpyAsync(d_base, h_base.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, st));
    GK_TRY(scr.alloc(rs, total + 1));
    GK_COUNT();
    k_globalize_rank<<<G(ctx, tot), 256, 0, st>>>(nsets, S, d_base, *rank);
    GK_COUNT();
    k_globalize_rs<<<dim3((unsigned)std::min<int64_t>(ceil_div(maxr, 256), 4096), S), 256, 0, st>>>(
        nsets, runs, d_base, rs_seg, *rs, S);
    GK_LAUNCH(ctx);
    *nbins = total;
    return GEEK_OK;
}

// Bins of the main SILK pass for S tables at once, by exact hashing of the
// signatures (no sort of all S * nsets signatures): only bins of >= 2 virtual
// buckets take part in the vote, and single-bucket bins matter only when
// their weight is >= 2 and the bucket has >= delta objects.  Returns the
// vote's bins (perm: virtual bucket per position, rank: bin per position, rs:
// bin starts, nbins; positions grouped by bin, bins in arbitrary order -- the
// seeds do not depend on bin order) and the single-bin buckets (singles).
// ns1 > 0: sets 0 .. ns1-1 hold one object each, single_of maps an object
// to its one-object set, and function kst[instance * kst_stride + t] of
// table t is injective on the instance's ids, so that no two one-object sets
// share a signature and each other set finds the one that shares its own
// (k_set_sig_marks); ns1 = 0: no such guarantee, every set goes through the
// seen maps and the grouping tables.
geek_status group_bins(geek_ctx *ctx, Scratch &scr, int S, int64_t nsets, const int64_t *soff, const uint32_t *sids,
                       int64_t nids, int64_t ns1, const uint8_t *kst, int kst_stride, const int32_t *single_of,
                       const int32_t *vw, int delta, int Ks, const uint64_t *A, const uint64_t *B, const SilkBatch *bt,
                       int64_t coef_stride, uint32_t **perm, int32_t **rank, int64_t **rs, int64_t *npos,
                       int64_t *nbins, int64_t **singles, int64_t *n_singles, cudaStream_t st) {
    const int64_t tot = (int64_t)S * nsets;
    const bool tagged = bt && bt->count > 1;
    // sets g0 .. nsets-1 go through the seen maps and the grouping tables;
    // one-object sets 0 .. ns1-1, on the claim path, are claimed by the sets
    // that share their signature (sets of many members take k_set_sig_sets
    // and no claims)
    const bool wide = nids >= SS_WIDE * nsets;
    const bool claims = ns1 > 0 && !wide && kst && single_of;
    const int64_t g0 = claims ? ns1 : 0, nm = nsets - g0;
    int64_t C = 64;
    while (C < 2 * nm) C <<= 1;
    const int64_t *roff = nullptr, *rcap = nullptr;
    if (tagged) {
        if (!bt->slot_off || !bt->slot_cap || !bt->slot_off_m || !bt->slot_cap_m)
            return set_error(ctx, GEEK_ERR_INVALID, "slot regions missing");
        roff = claims ? bt->slot_off_m : bt->slot_off;
        rcap = claims ? bt->slot_cap_m : bt->slot_cap;
        C = claims ? bt->slots_m : bt->slots;
    }
    uint64_t *klo, *khi = nullptr;
    if (nsets >= (int64_t)SLOT_MULTI - 1) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 2^31 SILK sets");
    uint32_t *tag = nullptr;
    uint64_t *slot;
    GK_TRY(scr.alloc(&klo, tot));
    if (Ks > 2) GK_TRY(scr.alloc(&khi, tot));
    if (tagged) GK_TRY(scr.alloc(&tag, tot));
    GK_TRY(scr.alloc(&slot, (size_t)S * C));
    GK_CUDA(ctx, cudaMemsetAsync(slot, 0xFF, sizeof(uint64_t) * S * C, st));
    uint64_t *mkey;
    uint32_t *mval;
    unsigned long long *counts;
    GK_TRY(scr.alloc(&mkey, tot));
    GK_TRY(scr.alloc(&mval, tot));
    GK_TRY(scr.alloc(singles, tot));
    GK_TRY(scr.alloc(&counts, 2));
    GK_CUDA(ctx, cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st));
    // seen-once / seen-twice maps: per table about four bits per set, at
    // most 2^28 bits (two parts of at most 32 MB)
    int64_t Mt = 1 << 10;
    while (Mt < 4 * nsets && Mt < ((int64_t)1 << 28)) Mt <<= 1;
    const int64_t M = Mt * S;
    uint32_t *seen;
    GK_TRY(scr.alloc(&seen, (size_t)(M / 32) * 2));
    GK_CUDA(ctx, cudaMemsetAsync(seen, 0, sizeof(uint32_t) * (size_t)(M / 32) * 2, st));
    uint32_t *seen1 = seen, *seen2 = seen + M / 32;
    const int gm = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nm, 256), (int64_t)ctx->num_sms * 8));
    const int gi = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nm, 256 * 4), (int64_t)ctx->num_sms * 8));
    static_assert(SM_U == 4 && GI_U == 4, "grid of the four-sets-per-thread kernels");
    int32_t *ms = nullptr;
    uint32_t *claimed = nullptr;
    const int64_t cwords = ceil_div(std::max<int64_t>(g0, 1), 32);
    if (claims) {
        GK_TRY(scr.alloc(&ms, std::max<int64_t>((int64_t)S * nm, 1)));
        GK_TRY(scr.alloc(&claimed, (size_t)S * cwords));
        GK_CUDA(ctx, cudaMemsetAsync(claimed, 0, sizeof(uint32_t) * (size_t)S * cwords, st));
    }
    if (nm > 0) {
        GK_COUNT();
        if (wide)
            k_set_sig_sets<<<gm, 256, 0, st>>>(nsets, S, soff, sids, Ks, A, B, tagged ? bt->row_off : nullptr,
                                               tagged ? bt->count : 1, tagged ? bt->set_inst : nullptr, coef_stride,
                                               klo, khi, nullptr, tag, seen1, seen2, (uint64_t)(Mt - 1), g0);
        else
            k_set_sig_marks<<<dim3(gi, S), 256, 0, st>>>(
                nsets, soff, sids, Ks, A, B, tagged ? bt->row_off : nullptr, tagged ? bt->count : 1,
                tagged ? bt->set_inst : nullptr, coef_stride, klo, khi, tag, seen1, seen2, (uint64_t)(Mt - 1), g0,
                kst, kst_stride, single_of, ms);
        GK_COUNT();
        k_group_insert<<<dim3(gi, S), 256, 0, st>>>(nsets, C, klo, khi, tag, roff, rcap, slot, mkey, mval, counts,
                                                    seen2, (uint64_t)(Mt - 1), vw, soff, delta, *singles, counts + 1,
                                                    g0, ms, claimed, cwords);
    }
    if (delta <= 1) {
        GK_COUNT();
        if (claims) {
            const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g0, 256), (int64_t)ctx->num_sms * 8));
            k_single_unclaimed<<<dim3(gs, S), 256, 0, st>>>(g0, claimed, cwords, vw, *singles, counts + 1);
        } else {
            k_group_singles<<<G(ctx, S * C), 256, 0, st>>>(C, S, slot, vw, soff, delta, *singles, counts + 1);
        }
    }
    GK_LAUNCH(ctx);
    unsigned long long h[2];
    GK_CUDA(ctx, cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    const int64_t m = (int64_t)h[0];
    *npos = m;
    *n_singles = (int64_t)h[1];
    // the vote's positions grouped by bin: sort the multi list by group key
    GK_TRY(radix_sort_segments(ctx, scr, 1, m, &mkey, nullptr, &mval, bit_length_u64((uint64_t)(S * C)), st));
    int64_t *runs;
    GK_TRY(scr.alloc(rank, std::max<int64_t>(m, 1)));
    GK_TRY(scr.alloc(rs, m + 1));
    GK_TRY(scr.alloc(&runs, 1));
    if (m > 0) {
        GK_TRY(segment_runs(ctx, scr, 1, m, mkey, nullptr, *rank, *rs, runs, st));
        GK_TRY(d2h_i64(ctx, runs, nbins, st));
    } else {
        *nbins = 0;
    }
    *perm = mval;
    return GEEK_OK;
}

// One slot region per instance for group_bins: a power of two >= 2x the
// instance's sets (device arrays from scr, total in bt->slots), and one sized
// for its sets from g_multi on (bt->slot_off_m ...: the claim path, on which
// only those sets enter the grouping tables).
geek_status slot_regions(geek_ctx *ctx, Scratch &scr, int64_t nsets, const int64_t *soff, const uint32_t *sids,
                         int64_t g_multi, SilkBatch *bt, cudaStream_t st) {
    const int count = bt->count;
    unsigned long long *cnt;
    uint32_t *set_inst;
    GK_TRY(scr.alloc(&cnt, 2 * (size_t)count));
    GK_TRY(scr.alloc(&set_inst, std::max<int64_t>(nsets, 1)));
    GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * count, st));
    if (nsets) {
        GK_COUNT();
        k_sets_per_inst<<<G(ctx, nsets), 256, 0, st>>>(nsets, soff, sids, bt->row_off, count, g_multi, cnt,
                                                       set_inst);
        GK_LAUNCH(ctx);
    }
    bt->set_inst = set_inst;
    std::vector<unsigned long long> hc(2 * (size_t)count);
    GK_CUDA(ctx, cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long) * hc.size(), cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int64_t> ho(2 * (size_t)count), hp(2 * (size_t)count);
    int64_t Cs[2] = {0, 0};
    for (int r = 0; r < 2; r++)
        for (int i = 0; i < count; i++) {
            int64_t c = 32;
            while (c < 2 * (int64_t)hc[(size_t)r * count + i]) c <<= 1;
            ho[(size_t)r * count + i] = Cs[r];
            hp[(size_t)r * count + i] = c;
            Cs[r] += c;
        }
    int64_t *roff, *rcap;
    GK_TRY(scr.alloc(&roff, 2 * (size_t)count));
    GK_TRY(scr.alloc(&rcap, 2 * (size_t)count));
    GK_CUDA(ctx, cudaMemcpyAsync(roff, ho.data(), sizeof(int64_t) * ho.size(), cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaMemcpyAsync(rcap, hp.data(), sizeof(int64_t) * hp.size(), cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));  // ho / hp leave scope
    bt->slot_off = roff;
    bt->slot_cap = rcap;
    bt->slots = Cs[0];
    bt->slot_off_m = roff + count;
    bt->slot_cap_m = rcap + count;
    bt->slots_m = Cs[1];
    return GEEK_OK;
}

// Majority vote of every bin holding >= 2 sets; bins whose C_shared has at
// least delta objects are emitted (ascending bin order, ascending ids).
// ok[b] tells which bins were emitted.
geek_status vote_bins(geek_ctx *ctx, Scratch &scr, int64_t m, const uint32_t *perm, const int32_t *rank,
                      const int64_t *rs, int64_t nbins, const int64_t *soff, const uint32_t *sids,
                      int delta, Csr *out, int64_t **ok_out, cudaStream_t st) {
    int64_t *w, *woff, *T_dev;
    GK_TRY(scr.alloc(&w, m));
    GK_TRY(scr.alloc(&woff, m));
    GK_TRY(scr.alloc(&T_dev, 1));
    GK_COUNT();
    k_vote_weights<<<G(ctx, m), 256, 0, st>>>(m, rank, rs, perm, soff, w);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, w, woff, m, T_dev, st));
    int64_t T = 0;
    GK_TRY(d2h_i64(ctx, T_dev, &T, st));
    int64_t *cnt, *ok, *len;
    GK_TRY(scr.alloc(&cnt, nbins));
    GK_TRY(scr.alloc(&ok, nbins));
    GK_TRY(scr.alloc(&len, nbins));
    GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * nbins, st));
    *ok_out = ok;
    out->n = 0;
    out->nids = 0;
    if (T == 0) {
        GK_CUDA(ctx, cudaMemsetAsync(ok, 0, sizeof(int64_t) * nbins, st));
        return GEEK_OK;
    }
    uint64_t *pairs;
    GK_TRY(scr.alloc(&pairs, T));
    GK_COUNT();
    k_vote_expand<<<G(ctx, m), 256, 0, st>>>(m, rank, perm, woff, w, soff, sids, pairs);
    GK_LAUNCH(ctx);
    const int nbits = 32 + bit_length_u64((uint64_t)nbins);
    GK_TRY(radix_sort_segments(ctx, scr, 1, T, &pairs, nullptr, nullptr, nbits, st));
    int64_t *prs, *nruns;
    GK_TRY(scr.alloc(&prs, T + 1));
    GK_TRY(scr.alloc(&nruns, 1));
    GK_TRY(segment_runs(ctx, scr, 1, T, pairs, nullptr, nullptr, prs, nruns, st));
    int64_t NR = 0;
    GK_TRY(d2h_i64(ctx, nruns, &NR, st));
    int64_t *keep, *sel, *pos, *total, *boffs, *set_idx, *nsets;
    GK_TRY(scr.alloc(&keep, NR));
    GK_TRY(scr.alloc(&sel, NR));
    GK_TRY(scr.alloc(&pos, NR));
    GK_TRY(scr.alloc(&total, 1));
    GK_TRY(scr.alloc(&boffs, nbins));
    GK_TRY(scr.alloc(&set_idx, nbins));
    GK_TRY(scr.alloc(&nsets, 1));
    GK_COUNT();
    k_vote_keep<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, rs, keep, cnt);
    GK_COUNT();
    k_bin_ok<<<G(ctx, nbins), 256, 0, st>>>(nbins, rs, cnt, delta, ok, len);
    GK_COUNT();
    k_vote_sel<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, keep, ok, sel);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, sel, pos, NR, total, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, len, boffs, nbins, nullptr, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, ok, set_idx, nbins, nsets, st));
    int64_t h_total = 0, h_nsets = 0;
    GK_TRY(d2h_i64(ctx, total, &h_total, st));
    GK_TRY(d2h_i64(ctx, nsets, &h_nsets, st));
    out->n = h_nsets;
    out->nids = h_total;
    GK_TRY(scr.alloc(&out->off, h_nsets + 1));
    GK_TRY(scr.alloc(&out->ids, std::max<int64_t>(1, h_total)));
    GK_COUNT();
    k_vote_emit<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, sel, pos, out->ids);
    GK_COUNT();
    k_compact_offsets<<<G(ctx, nbins), 256, 0, st>>>(nbins, ok, set_idx, boffs, out->off, nsets, total);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

// Weighted majority vote of every bin holding >= 2 virtual buckets; emits
// C_shared of the bins whose vote has at least delta objects.
geek_status wvote_bins(geek_ctx *ctx, Scratch &scr, int64_t m, const uint32_t *perm, const int32_t *rank,
                       const int64_t *rs, int64_t nbins, const int64_t *voff, const uint32_t *vmem,
                       const int32_t *vw, const int64_t *bw, int delta, Csr *out, cudaStream_t st) {
    int64_t *w, *woff, *T_dev;
    uint8_t *pruned;
    GK_TRY(scr.alloc(&w, m));
    GK_TRY(scr.alloc(&woff, m));
    GK_TRY(scr.alloc(&T_dev, 1));
    GK_TRY(scr.alloc(&pruned, nbins));
    GK_COUNT();
    k_bin_prune<<<G(ctx, nbins), 256, 0, st>>>(nbins, rs, perm, vw, voff, bw, delta, pruned);
    GK_COUNT();
    k_wvote_weights<<<G(ctx, m), 256, 0, st>>>(m, rank, rs, perm, voff, pruned, w);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, w, woff, m, T_dev, st));
    int64_t T = 0;
    GK_TRY(d2h_i64(ctx, T_dev, &T, st));
    out->n = 0;
    out->nids = 0;
    if (T == 0) return GEEK_OK;
    uint64_t *pairs;
    uint32_t *pw;
    GK_TRY(scr.alloc(&pairs, T));
    GK_TRY(scr.alloc(&pw, T));
    GK_COUNT();
    k_wvote_expand<<<G(ctx, m), 256, 0, st>>>(m, rank, perm, woff, w, voff, vmem, vw, pairs, pw);
    GK_LAUNCH(ctx);
    GK_TRY(radix_sort_segments(ctx, scr, 1, T, &pairs, nullptr, &pw, 32 + bit_length_u64((uint64_t)nbins), st));
    int64_t *prs, *nruns;
    GK_TRY(scr.alloc(&prs, T + 1));
    GK_TRY(scr.alloc(&nruns, 1));
    GK_TRY(segment_runs(ctx, scr, 1, T, pairs, nullptr, nullptr, prs, nruns, st));
    int64_t NR = 0;
    GK_TRY(d2h_i64(ctx, nruns, &NR, st));
    int64_t *keep, *sel, *pos, *total, *boffs, *set_idx, *nsets, *cnt, *ok, *len;
    GK_TRY(scr.alloc(&keep, NR));
    GK_TRY(scr.alloc(&sel, NR));
    GK_TRY(scr.alloc(&pos, NR));
    GK_TRY(scr.alloc(&total, 1));
    GK_TRY(scr.alloc(&boffs, nbins));
    GK_TRY(scr.alloc(&set_idx, nbins));
    GK_TRY(scr.alloc(&nsets, 1));
    GK_TRY(scr.alloc(&cnt, nbins));
    GK_TRY(scr.alloc(&ok, nbins));
    GK_TRY(scr.alloc(&len, nbins));
    GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * nbins, st));
    GK_COUNT();
    k_wvote_keep<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, pw, bw, keep, cnt);
    GK_COUNT();
    k_wbin_ok<<<G(ctx, nbins), 256, 0, st>>>(nbins, rs, cnt, delta, ok, len);
    GK_COUNT();
    k_vote_sel<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, keep, ok, sel);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, sel, pos, NR, total, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, len, boffs, nbins, nullptr, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, ok, set_idx, nbins, nsets, st));
    int64_t h_total = 0, h_nsets = 0;
    GK_TRY(d2h_i64(ctx, total, &h_total, st));
    GK_TRY(d2h_i64(ctx, nsets, &h_nsets, st));
    out->n = h_nsets;
    out->nids = h_total;
    GK_TRY(scr.alloc(&out->off, h_nsets + 1));
    GK_TRY(scr.alloc(&out->ids, std::max<int64_t>(1, h_total)));
    GK_COUNT();
    k_vote_emit<<<G(ctx, NR), 256, 0, st>>>(nruns, prs, pairs, sel, pos, out->ids);
    GK_COUNT();
    k_compact_offsets<<<G(ctx, nbins), 256, 0, st>>>(nbins, ok, set_idx, boffs, out->off, nsets, total);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

// gathers the listed sets (device index list) into a new CSR
geek_status gather_sets(geek_ctx *ctx, Scratch &scr, int64_t cnt, const int64_t *idx,
                        const int64_t *soff, const uint32_t *sids, Csr *out, cudaStream_t st) {
    out->n = cnt;
    int64_t *len, *tot;
    GK_TRY(scr.alloc(&len, std::max<int64_t>(cnt, 1)));
    GK_TRY(scr.alloc(&out->off, cnt + 1));
    GK_TRY(scr.alloc(&tot, 1));
    GK_COUNT();
    k_gather_len<<<G(ctx, cnt), 256, 0, st>>>(cnt, idx, soff, len);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, len, out->off, cnt, tot, st));
    GK_CUDA(ctx, cudaMemcpyAsync(out->off + cnt, tot, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    GK_TRY(d2h_i64(ctx, tot, &out->nids, st));
    GK_TRY(scr.alloc(&out->ids, std::max<int64_t>(1, out->nids)));
    GK_COUNT();
    k_gather_ids<<<G(ctx, cnt), 256, 0, st>>>(cnt, idx, soff, sids, out->off, out->ids);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

// concatenation of CSR pieces
geek_status concat_sets(geek_ctx *ctx, Scratch &scr, const std::vector<Csr> &parts, Csr *out,
                        cudaStream_t st) {
    int64_t n = 0, nids = 0;
    for (auto &p : parts) {
        n += p.n;
        nids += p.nids;
    }
    out->n = n;
    out->nids = nids;
    GK_TRY(scr.alloc(&out->off, n + 1));
    GK_TRY(scr.alloc(&out->ids, std::max<int64_t>(1, nids)));
    // offsets: copy each part's offsets shifted by the running id count
    std::vector<int64_t> h_off;
    h_off.reserve(n + 1);
    int64_t base = 0, ibase = 0;
    for (auto &p : parts) {
        if (p.n == 0) continue;
        std::vector<int64_t> tmp(p.n + 1);
        GK_CUDA(ctx, cudaMemcpyAsync(tmp.data(), p.off, sizeof(int64_t) * (p.n + 1), cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        for (int64_t i = 0; i < p.n; i++) h_off.push_back(tmp[i] + ibase);
        if (p.nids)
            GK_CUDA(ctx, cudaMemcpyAsync(out->ids + ibase, p.ids, sizeof(uint32_t) * p.nids, cudaMemcpyDeviceToDevice, st));
        ibase += p.nids;
        base += p.n;
    }
    h_off.push_back(ibase);
    GK_CUDA(ctx, cudaMemcpyAsync(out->off, h_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    (void)base;
    return GEEK_OK;
}

}  // namespace

geek_status silk_run(geek_ctx *ctx, const geek_buckets *b, const silk_params *p, silk_seeds *out,
                     cudaStream_t st, const SilkBatch *bt) {
    Scratch scr(ctx, st);
    const int Ks = p->Ks, Ls = p->Ls, delta = p->delta;
    const int64_t NB = b->NB;
    std::vector<Csr> parts;
    // ---- virtual buckets (see k_vb_count) -------------------------------------
    EvTimer t_vb(ctx, "silk.vbuckets", st);
    const int64_t n = b->n;
    int32_t *mult;
    int64_t *ns_flag, *s_flag, *s_pos, *n_pos, *d_ns1, *d_ns2;
    GK_TRY(scr.alloc(&mult, std::max<int64_t>(n, 1)));
    GK_TRY(scr.alloc(&ns_flag, std::max<int64_t>(NB, 1)));
    GK_TRY(scr.alloc(&s_flag, std::max<int64_t>(n, 1)));
    GK_TRY(scr.alloc(&s_pos, std::max<int64_t>(n, 1)));
    GK_TRY(scr.alloc(&n_pos, std::max<int64_t>(NB, 1)));
    GK_TRY(scr.alloc(&d_ns1, 1));
    GK_TRY(scr.alloc(&d_ns2, 1));
    GK_CUDA(ctx, cudaMemsetAsync(mult, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    GK_COUNT();
    k_vb_count<<<G(ctx, NB), 256, 0, st>>>(NB, b->boff, b->members, mult, ns_flag);
    GK_COUNT();
    k_pos_flag<<<G(ctx, n), 256, 0, st>>>(n, mult, s_flag);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, s_flag, s_pos, n, d_ns1, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, ns_flag, n_pos, NB, d_ns2, st));
    int64_t NS1 = 0, NS2 = 0;
    GK_TRY(d2h_i64(ctx, d_ns1, &NS1, st));
    GK_TRY(d2h_i64(ctx, d_ns2, &NS2, st));
    const int64_t NV = NS1 + NS2;
    int64_t *vsz, *vsrc, *voff, *d_vtot;
    int32_t *vw, *single_of;
    uint32_t *vmem;
    GK_TRY(scr.alloc(&single_of, std::max<int64_t>(n, 1)));
    GK_TRY(scr.alloc(&vsz, std::max<int64_t>(NV, 1)));
    GK_TRY(scr.alloc(&vsrc, std::max<int64_t>(NV, 1)));
    GK_TRY(scr.alloc(&vw, std::max<int64_t>(NV, 1)));
    GK_TRY(scr.alloc(&voff, NV + 1));
    GK_TRY(scr.alloc(&d_vtot, 1));
    GK_COUNT();
    k_vb_fill_s<<<G(ctx, n), 256, 0, st>>>(n, mult, s_pos, vsz, vw, vsrc, single_of);
    GK_COUNT();
    k_vb_fill_n<<<G(ctx, NB), 256, 0, st>>>(NB, b->boff, ns_flag, n_pos, NS1, vsz, vw, vsrc);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, vsz, voff, NV, d_vtot, st));
    GK_CUDA(ctx, cudaMemcpyAsync(voff + NV, d_vtot, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    int64_t VT = 0;
    GK_TRY(d2h_i64(ctx, d_vtot, &VT, st));
    GK_TRY(scr.alloc(&vmem, std::max<int64_t>(VT, 1)));
    GK_COUNT();
    k_vb_members<<<G(ctx, NV), 256, 0, st>>>(NV, NS1, vsrc, voff, b->boff, b->members, vmem);
    GK_LAUNCH(ctx);
    // SILK tables in which no two one-object virtual buckets can share a
    // signature: in every instance one of the table's Ks functions is
    // injective on the instance's ids (k_mh_injective); kst holds the first
    // such function per (instance, table), 255 where there is none
    std::vector<char> tab_one(Ls, 0);
    uint8_t *kst = nullptr;
    if (NS1 > 0) {
        const int cnt = (bt && bt->count > 1) ? bt->count : 1;
        uint32_t *fb;
        GK_TRY(scr.alloc(&fb, (size_t)cnt * Ls));
        GK_CUDA(ctx, cudaMemsetAsync(fb, 0, sizeof(uint32_t) * (size_t)cnt * Ls, st));
        GK_COUNT();
        k_mh_injective<<<G(ctx, n), 256, 0, st>>>(n, cnt > 1 ? bt->row_off : nullptr, cnt, p->mh_a,
                                                  (int64_t)Ls * Ks, Ls, Ks, fb);
        GK_LAUNCH(ctx);
        std::vector<uint32_t> hfb((size_t)cnt * Ls);
        GK_CUDA(ctx, cudaMemcpyAsync(hfb.data(), fb, sizeof(uint32_t) * hfb.size(), cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        std::vector<uint8_t> hk((size_t)cnt * Ls, 255);
        for (size_t e = 0; e < hk.size(); e++)
            for (int k = Ks - 1; k >= 0; k--)
                if (!((hfb[e] >> k) & 1u)) hk[e] = (uint8_t)k;
        for (int t = 0; t < Ls; t++) {
            bool ok = true;
            for (int i = 0; i < cnt && ok; i++) ok = hk[(size_t)i * Ls + t] != 255;
            tab_one[t] = ok;
        }
        GK_TRY(scr.alloc(&kst, hk.size()));
        GK_CUDA(ctx, cudaMemcpyAsync(kst, hk.data(), hk.size(), cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
    }

    t_vb.stop();
    SilkBatch btl;  // batched: per-instance slot regions of the grouping tables
    if (bt && bt->count > 1) {
        btl = *bt;
        GK_TRY(slot_regions(ctx, scr, NV, voff, vmem, NS1, &btl, st));
        bt = &btl;
    }
    // ---- Alg. 4: Ls SILK tables over the (virtual) buckets ------------------
    // SILK tables are processed in chunks of S (all at once when they fit the
    // position budget); bins of a chunk are numbered globally
    const int64_t budget = (int64_t)1 << 27;
    const int TS = (int)std::max<int64_t>(1, std::min<int64_t>(Ls, NV > 0 ? budget / NV : Ls));
    for (int t = 0; t < Ls && NV > 0; t += TS) {
        const int S = std::min(TS, Ls - t);
        Scratch tscr(ctx, st);  // per-chunk temporaries
        uint32_t *perm;
        int32_t *rank;
        int64_t *rs, nbins = 0, *singles, nh = 0, npos = 0;
        bool one = true;
        for (int u = t; u < t + S; u++) one = one && tab_one[u];
        {
            EvTimer tb(ctx, "silk.bins", st);
            GK_TRY(group_bins(ctx, tscr, S, NV, voff, vmem, VT, one ? NS1 : 0, kst ? kst + t : nullptr, Ls,
                              single_of, vw, delta, Ks, p->mh_a + (int64_t)t * Ks,
                              p->mh_b + (int64_t)t * Ks, bt, (int64_t)Ls * Ks, &perm, &rank, &rs, &npos, &nbins,
                              &singles, &nh, st));
        }
        EvTimer tv(ctx, "silk.vote", st);
        int64_t *bw;
        GK_TRY(tscr.alloc(&bw, std::max<int64_t>(nbins, 1)));
        if (nbins) {
            GK_COUNT();
            k_bin_weight<<<G(ctx, nbins), 256, 0, st>>>(nbins, rs, perm, vw, bw);
            GK_LAUNCH(ctx);
        }
        std::vector<Csr> tparts;
        if (nh) {
            Csr c1;
            GK_TRY(gather_sets(ctx, tscr, nh, singles, voff, vmem, &c1, st));
            tparts.push_back(c1);
        }
        Csr c2;
        if (nbins) GK_TRY(wvote_bins(ctx, tscr, npos, perm, rank, rs, nbins, voff, vmem, vw, bw, delta, &c2, st));
        if (c2.n) tparts.push_back(c2);
        for (auto &c : tparts) {
            // move the table's C_shared sets into the outer scratch
            Csr keep;
            keep.n = c.n;
            keep.nids = c.nids;
            GK_TRY(scr.alloc(&keep.off, c.n + 1));
            GK_TRY(scr.alloc(&keep.ids, std::max<int64_t>(1, c.nids)));
            GK_CUDA(ctx, cudaMemcpyAsync(keep.off, c.off, sizeof(int64_t) * (c.n + 1), cudaMemcpyDeviceToDevice, st));
            if (c.nids)
                GK_CUDA(ctx, cudaMemcpyAsync(keep.ids, c.ids, sizeof(uint32_t) * c.nids, cudaMemcpyDeviceToDevice, st));
            parts.push_back(keep);
        }
        GK_CUDA(ctx, cudaStreamSynchronize(st));
    }
    Csr C;
    GK_TRY(concat_sets(ctx, scr, parts, &C, st));
    out->n_multiset = C.n;

    // ---- near-duplicate removal: one more table over C --------------------
    EvTimer t_dd(ctx, "silk.dedup", st);
    std::vector<Csr> dparts;
    if (C.n > 0) {
        uint32_t *perm;
        int32_t *rank;
        int64_t *rs, nbins = 0;
        GK_TRY(make_bins(ctx, scr, 1, C.n, C.off, C.ids, C.nids, Ks, p->dd_a, p->dd_b, bt, Ks, &perm, &rank, &rs, &nbins,
                         st));
        Csr V;
        int64_t *ok;
        GK_TRY(vote_bins(ctx, scr, C.n, perm, rank, rs, nbins, C.off, C.ids, delta, &V, &ok, st));
        if (V.n) dparts.push_back(V);
        int64_t *pick, *has, *pos, *npick;
        GK_TRY(scr.alloc(&pick, nbins));
        GK_TRY(scr.alloc(&has, nbins));
        GK_TRY(scr.alloc(&pos, nbins));
        GK_TRY(scr.alloc(&npick, 1));
        GK_COUNT();
        k_dedup_pick<<<G(ctx, nbins), 256, 0, st>>>(nbins, rs, perm, ok, C.off, C.ids, pick, has);
        GK_LAUNCH(ctx);
        GK_TRY(exclusive_scan_i64(ctx, scr, has, pos, nbins, npick, st));
        int64_t hp = 0;
        GK_TRY(d2h_i64(ctx, npick, &hp, st));
        if (hp) {
            int64_t *idx;
            GK_TRY(scr.alloc(&idx, hp));
            GK_COUNT();
            k_compact_idx<<<G(ctx, nbins), 256, 0, st>>>(nbins, has, pos, pick, idx);
            GK_LAUNCH(ctx);
            Csr P;
            GK_TRY(gather_sets(ctx, scr, hp, idx, C.off, C.ids, &P, st));
            dparts.push_back(P);
        }
    }
    Csr D;
    GK_TRY(concat_sets(ctx, scr, dparts, &D, st));

    // ---- canonical order, exact duplicates out -----------------------------
    out->k = 0;
    out->n_ids = 0;
    if (D.n == 0) {
        GK_CUDA(ctx, cudaMallocAsync((void **)&out->off, sizeof(int64_t), st));
        GK_CUDA(ctx, cudaMemsetAsync(out->off, 0, sizeof(int64_t), st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        return GEEK_OK;
    }
    uint64_t *key;
    uint32_t *perm;
    GK_TRY(scr.alloc(&key, D.n));
    GK_TRY(scr.alloc(&perm, D.n));
    GK_COUNT();
    k_prefix_key<<<G(ctx, D.n), 256, 0, st>>>(D.n, D.off, D.ids, key, perm);
    GK_LAUNCH(ctx);
    GK_TRY(radix_sort_segments(ctx, scr, 1, D.n, &key, nullptr, &perm, 64, st));
    int32_t *rank;
    int64_t *rs, *nr, *order, *keep, *kpos, *kt;
    GK_TRY(scr.alloc(&rank, D.n));
    GK_TRY(scr.alloc(&rs, D.n + 1));
    GK_TRY(scr.alloc(&nr, 1));
    GK_TRY(segment_runs(ctx, scr, 1, D.n, key, nullptr, rank, rs, nr, st));
    GK_TRY(scr.alloc(&order, D.n));
    GK_TRY(scr.alloc(&keep, D.n));
    GK_TRY(scr.alloc(&kpos, D.n));
    GK_TRY(scr.alloc(&kt, 1));
    GK_COUNT();
    k_prefix_fix<<<G(ctx, D.n), 256, 0, st>>>(D.n, rank, rs, perm, D.off, D.ids, order);
    GK_COUNT();
    k_dup_flags<<<G(ctx, D.n), 256, 0, st>>>(D.n, order, D.off, D.ids, keep);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, keep, kpos, D.n, kt, st));
    int64_t k = 0;
    GK_TRY(d2h_i64(ctx, kt, &k, st));
    int64_t *sel;
    GK_TRY(scr.alloc(&sel, k));
    GK_COUNT();
    k_compact_idx<<<G(ctx, D.n), 256, 0, st>>>(D.n, keep, kpos, order, sel);
    GK_LAUNCH(ctx);
    Csr E;
    GK_TRY(gather_sets(ctx, scr, k, sel, D.off, D.ids, &E, st));
    // hand the final CSR to the handle (persistent allocations)
    GK_CUDA(ctx, cudaMallocAsync((void **)&out->off, sizeof(int64_t) * (k + 1), st));
    GK_CUDA(ctx, cudaMallocAsync((void **)&out->ids, sizeof(int32_t) * std::max<int64_t>(1, E.nids), st));
    GK_CUDA(ctx, cudaMemcpyAsync(out->off, E.off, sizeof(int64_t) * (k + 1), cudaMemcpyDeviceToDevice, st));
    if (E.nids)
        GK_CUDA(ctx, cudaMemcpyAsync(out->ids, E.ids, sizeof(uint32_t) * E.nids, cudaMemcpyDeviceToDevice, st));
    int sort_err = 0;
    GK_TRY(sort_err_fetch(ctx, &sort_err, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    GK_TRY(sort_err_eval(ctx, &sort_err, st));
    out->k = k;
    out->n_ids = E.nids;
    return GEEK_OK;
}
