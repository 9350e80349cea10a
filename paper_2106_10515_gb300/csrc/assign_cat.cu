// Central vectors and assignment for categorical and set data (Sect. 3.3):
//  - heterogeneous rows: unified categorical attributes (per table, the
//    packed key of the numeric E2LSH part; then the tokens), per-attribute
//    mode as central vector, distance 1 - Jaccard = most matching attributes;
//  - sparse sets: central vector = items present in more than half of the
//    members, distance 1 - |A n C| / |A u C| compared exactly as fractions.
#include <algorithm>

#include "internal.cuh"

namespace {

int G(geek_ctx *ctx, int64_t work) { return grid_for(std::max<int64_t>(work, 1), 256, ctx->num_sms); }

// attrs[i][a]: a < L -> numeric key of table a, else token a - L
__global__ void k_build_attrs(int64_t n, int L, int ncat, const uint64_t *__restrict__ num_key,
                              const uint32_t *__restrict__ tok, uint64_t *__restrict__ attrs) {
    const int A = L + ncat;
    const int64_t total = n * A;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / A;
        const int a = (int)(e % A);
        attrs[e] = a < L ? num_key[(int64_t)a * n + i] : (uint64_t)tok[i * ncat + (a - L)];
    }
}

// mode of attribute a over seed j's members: most frequent value, ties to the
// smallest (one thread per (seed, attribute); quadratic in the seed size)
// rep (nullable): the first member, in the seed's ascending order, holding
// the mode value
__global__ void k_modes(int64_t k, int A, const int64_t *__restrict__ soff, const int32_t *__restrict__ sids,
                        const uint64_t *__restrict__ attrs, uint64_t *__restrict__ modes, int32_t *__restrict__ rep) {
    const int64_t total = k * A;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / A;
        const int a = (int)(e % A);
        const int64_t s = soff[j], t = soff[j + 1];
        uint64_t best = 0;
        int64_t bc = 0;
        int32_t br = -1;
        for (int64_t p = s; p < t; p++) {
            const uint64_t v = attrs[(int64_t)sids[p] * A + a];
            int64_t c = 0;
            for (int64_t q = s; q < t; q++) c += attrs[(int64_t)sids[q] * A + a] == v;
            if (c > bc || (c == bc && v < best)) {
                bc = c;
                best = v;
                br = sids[p];
            }
        }
        modes[e] = best;
        if (rep) rep[e] = br;
    }
}

// flags[g] = 1 where bucket g (global id, in table l's canonical order) starts
// a new numeric E2LSH tuple: the table keys of heterogeneous rows put the
// numeric tuple first, so equal numeric tuples form runs of buckets.
__global__ void k_num_run_flags(int64_t nb, int64_t base, const int64_t *__restrict__ boff,
                                const uint32_t *__restrict__ members, const uint64_t *__restrict__ num_key_l,
                                int64_t *__restrict__ flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nb; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = base + r;
        int64_t f = 1;
        if (r > 0) f = num_key_l[members[boff[g]]] != num_key_l[members[boff[g - 1]]];
        flags[g] = f;
    }
}

// modes as a user sees them: per table, the rank of the mode's numeric tuple
// among the table's distinct numeric tuples (via the bucket of the member
// that holds it); then the mode tokens
__global__ void k_mode_out(int64_t k, int A, int L, int64_t n, const uint64_t *__restrict__ modes,
                           const int32_t *__restrict__ rep, const int32_t *__restrict__ obj_bucket,
                           const int64_t *__restrict__ tbase, const int64_t *__restrict__ excl,
                           const int64_t *__restrict__ flags, int64_t *__restrict__ out) {
    const int64_t total = k * A;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % A);
        if (a < L) {
            // runs started at or before g, less the one at the table's start
            const int64_t g = tbase[a] + obj_bucket[(int64_t)a * n + rep[e]];
            out[e] = excl[g] + flags[g] - 1 - excl[tbase[a]];
        } else {
            out[e] = (int64_t)modes[e];
        }
    }
}

// label = argmax_j #{a : attrs[i][a] == modes[j][a]}, ties to the smallest j
constexpr int CAT_TILE = 64;
constexpr int CAT_MAXA = 32;
__global__ void __launch_bounds__(256) k_assign_cat(int64_t n, int A, int64_t k, const uint64_t *__restrict__ attrs,
                                                    const uint64_t *__restrict__ modes, int32_t *__restrict__ labels,
                                                    int32_t *__restrict__ matches) {
    __shared__ uint64_t ms[CAT_TILE * CAT_MAXA];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x[CAT_MAXA];
    for (int a = 0; a < CAT_MAXA; a++) x[a] = (i < n && a < A) ? attrs[i * A + a] : 0;
    int bm = -1, bj = -1;
    for (int64_t j0 = 0; j0 < k; j0 += CAT_TILE) {
        __syncthreads();
        const int tn = (int)min((int64_t)CAT_TILE, k - j0);
        for (int e = threadIdx.x; e < tn * A; e += blockDim.x) ms[(e / A) * CAT_MAXA + e % A] = modes[(j0 + e / A) * A + e % A];
        __syncthreads();
        for (int jj = 0; jj < tn; jj++) {
            int m = 0;
#pragma unroll
            for (int a = 0; a < CAT_MAXA; a++)
                if (a < A) m += x[a] == ms[jj * CAT_MAXA + a];
            if (m > bm) {
                bm = m;
                bj = (int)(j0 + jj);
            }
        }
    }
    if (i < n) {
        labels[i] = bj;
        if (matches) matches[i] = bm;
    }
}

// ---- set data --------------------------------------------------------------

// member weight of each (group, member) entry = size of the member's set
__global__ void k_group_w(int64_t m, const int32_t *__restrict__ gmem, const int64_t *__restrict__ soff,
                          int64_t *__restrict__ w) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        w[p] = soff[gmem[p] + 1] - soff[gmem[p]];
}

__global__ void k_group_of(int64_t ng, const int64_t *__restrict__ goff, int32_t *__restrict__ gid) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = goff[g]; p < goff[g + 1]; p++) gid[p] = (int32_t)g;
}

__global__ void k_group_expand(int64_t m, const int32_t *__restrict__ gid, const int32_t *__restrict__ gmem,
                               const int64_t *__restrict__ woff, const int64_t *__restrict__ soff,
                               const uint32_t *__restrict__ sids, uint64_t *__restrict__ pairs) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t g = (uint64_t)gid[p];
        const int32_t s = gmem[p];
        int64_t o = woff[p];
        for (int64_t q = soff[s]; q < soff[s + 1]; q++) pairs[o++] = (g << 32) | sids[q];
    }
}

__global__ void k_group_keep(const int64_t *__restrict__ nruns, const int64_t *__restrict__ prs,
                             const uint64_t *__restrict__ pairs, const int64_t *__restrict__ goff,
                             int64_t *__restrict__ keep, int64_t *__restrict__ cnt) {
    const int64_t nr = *nruns;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = prs[r + 1] - prs[r];
        const int64_t g = (int64_t)(pairs[prs[r]] >> 32);
        const bool kp = 2 * len > goff[g + 1] - goff[g];
        keep[r] = kp;
        if (kp) atomicAdd((unsigned long long *)&cnt[g], 1ull);
    }
}

__global__ void k_group_emit(const int64_t *__restrict__ nruns, const int64_t *__restrict__ prs,
                             const uint64_t *__restrict__ pairs, const int64_t *__restrict__ keep,
                             const int64_t *__restrict__ pos, uint32_t *__restrict__ out) {
    const int64_t nr = *nruns;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x)
        if (keep[r]) out[pos[r]] = (uint32_t)(pairs[prs[r]] & 0xFFFFFFFFu);
}

// heavy items: up to 64 * JX_HW of the items with the longest posting lists
// are counted by bitmasks instead of posting lists
constexpr int JX_HW = 1;

// item -> centres inverted index helpers
__global__ void k_centre_pairs(int64_t k, const int64_t *__restrict__ coff, const uint32_t *__restrict__ citems,
                               uint64_t *__restrict__ pairs) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = coff[j]; p < coff[j + 1]; p++) pairs[p] = ((uint64_t)citems[p] << 32) | (uint64_t)j;
}


__global__ void k_item_key(int64_t m, const uint64_t *__restrict__ pairs, uint64_t *__restrict__ ikey) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x)
        ikey[q] = pairs[q] >> 32;
}



__global__ void k_light_flags(int64_t nr, const int64_t *__restrict__ rs, const int64_t *__restrict__ is_heavy,
                              int64_t *__restrict__ lrun, int64_t *__restrict__ lent) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
        const bool light = !is_heavy[r];
        lrun[r] = light;
        lent[r] = light ? rs[r + 1] - rs[r] : 0;
    }
}

__global__ void k_light_emit(int64_t nr, const int64_t *__restrict__ rs, const uint64_t *__restrict__ ikey,
                             const uint64_t *__restrict__ pairs, const int64_t *__restrict__ is_heavy,
                             const int64_t *__restrict__ lrun_pos, const int64_t *__restrict__ lent_pos,
                             uint32_t *__restrict__ litem, int64_t *__restrict__ loff, uint32_t *__restrict__ lcentre,
                             const int64_t *__restrict__ nlent, int64_t nlight) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
        if (is_heavy[r]) continue;
        const int64_t p = lrun_pos[r];
        litem[p] = (uint32_t)ikey[rs[r]];
        loff[p] = lent_pos[r];
        int64_t o = lent_pos[r];
        for (int64_t q = rs[r]; q < rs[r + 1]; q++) lcentre[o++] = (uint32_t)(pairs[q] & 0xFFFFFFFFu);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) loff[nlight] = *nlent;
}

__global__ void k_iota_rows(int64_t n, int32_t *__restrict__ rows, unsigned long long *__restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rows[i] = (int32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = (unsigned long long)n;
}

// item of each listed run (first entry's key)
__global__ void k_run_items(int nh, const int64_t *__restrict__ runs, const int64_t *__restrict__ rs,
                            const uint64_t *__restrict__ ikey, uint32_t *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nh; q += gridDim.x * blockDim.x)
        out[q] = (uint32_t)ikey[rs[runs[q]]];
}

// heavy items: bit b of the HW-word mask stands for the item hv_item[i] with
// hv_bit[i] = b (hv_item ascending); -1 when x is not heavy
__device__ __forceinline__ int heavy_bit(uint32_t x, const uint32_t *__restrict__ hv_item,
                                         const int16_t *__restrict__ hv_bit, int nheavy) {
    int lo = 0, hi = nheavy;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (hv_item[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return (lo < nheavy && hv_item[lo] == x) ? hv_bit[lo] : -1;
}

__global__ void k_heavy_masks(int64_t k, const int64_t *__restrict__ coff, const uint32_t *__restrict__ citems,
                              const uint32_t *__restrict__ hv_item, const int16_t *__restrict__ hv_bit, int nheavy,
                              int HW, uint64_t *__restrict__ cmask, int32_t *__restrict__ clen) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t m[JX_HW] = {};
        for (int64_t p = coff[j]; p < coff[j + 1]; p++) {
            const int b = heavy_bit(citems[p], hv_item, hv_bit, nheavy);
            if (b >= 0) m[b >> 6] |= 1ull << (b & 63);
        }
        for (int w = 0; w < HW; w++) cmask[j * HW + w] = m[w];
        clen[j] = (int32_t)(coff[j + 1] - coff[j]);
    }
}

// Jaccard assignment: warp per set.  Intersections with heavy items come
// from bitmasks; light items go through the inverted index into a per-warp
// counter array (cleared after use).  Every centre is then scored exactly:
// J_j = inter / (|A| + |C_j| - inter), compared by cross-multiplication.
// (The dense path: every centre is scanned per set.  It serves the sets
// whose light candidates overflow the shared-memory table of k_jac_light;
// rows lists them, na_fix >= 0 replaces |A| by a fixed size.)
__global__ void __launch_bounds__(256) k_assign_jaccard(
    int64_t n, const int64_t *__restrict__ off, const uint32_t *__restrict__ items, int64_t k,
    const int32_t *__restrict__ clen, const uint64_t *__restrict__ cmask, const uint32_t *__restrict__ hv_item,
    const int16_t *__restrict__ hv_bit, int nheavy, int HW, const uint32_t *__restrict__ post_item,
    const int64_t *__restrict__ post_off, int64_t n_post_items, const uint32_t *__restrict__ post_centre,
    int32_t *__restrict__ counts, int32_t *__restrict__ labels, const int32_t *__restrict__ rows,
    const unsigned long long *__restrict__ n_rows, int na_fix) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t *cnt = counts + warp * k;
    if (rows) n = (int64_t)*n_rows;
    for (int64_t ii = warp; ii < n; ii += nw) {
        const int64_t i = rows ? (int64_t)rows[ii] : ii;
        const int64_t s = off[i], e = off[i + 1];
        const int64_t na = na_fix >= 0 ? na_fix : e - s;
        uint64_t am[JX_HW] = {};
        // light items: binary search in the sorted item list of the index
        for (int64_t p = s + lane; p < e; p += 32) {
            const uint32_t it = items[p];
            const int hb = heavy_bit(it, hv_item, hv_bit, nheavy);
            if (hb >= 0) {
                am[hb >> 6] |= 1ull << (hb & 63);
                continue;
            }
            int64_t lo = 0, hi = n_post_items;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (post_item[mid] < it) lo = mid + 1;
                else hi = mid;
            }
            if (lo < n_post_items && post_item[lo] == it)
                for (int64_t q = post_off[lo]; q < post_off[lo + 1]; q++) atomicAdd(&cnt[post_centre[q]], 1);
        }
#pragma unroll
        for (int w = 0; w < JX_HW; w++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) am[w] |= __shfl_xor_sync(0xffffffffu, am[w], o);
        __syncwarp();
        __threadfence_block();
        int64_t bn = -1, bd = 1;
        int bj = 0x7FFFFFFF;
        for (int64_t j = lane; j < k; j += 32) {
            int64_t in = cnt[j];
            for (int w = 0; w < HW; w++) in += __popcll(am[w] & cmask[j * HW + w]);
            cnt[j] = 0;
            const int64_t un = na + clen[j] - in;
            const int64_t num = un ? in : 0, den = un ? un : 1;
            if (bj == 0x7FFFFFFF || num * bd > bn * den) {
                bn = num;
                bd = den;
                bj = (int)j;
            }
        }
        // warp argmax: larger fraction, then smaller index
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t on = __shfl_xor_sync(0xffffffffu, bn, o);
            const int64_t od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            bool take;
            if (oj == 0x7FFFFFFF) take = false;
            else if (bj == 0x7FFFFFFF) take = true;
            else {
                const int64_t l = on * bd, r = bn * od;
                take = l > r || (l == r && oj < bj);
            }
            if (take) {
                bn = on;
                bd = od;
                bj = oj;
            }
        }
        if (lane == 0) labels[i] = bj == 0x7FFFFFFF ? -1 : bj;
        __syncwarp();
    }
}

// Exact Jaccard argmax, tiled over the centres.  A block takes JX_S sets
// (one warp each) and walks the centres in tiles of KT; per tile, every
// item of a set reads the part of its posting list (centres containing the
// item, ascending) that falls in the tile, found from precomputed per-tile
// offsets, and adds one to the set's counter of each centre there (packed
// 8- or 16-bit counters in shared memory: a counter counts the set's light
// items in one centre, at most the variant's MAXI).  The counters are
// then |A n C_j| for every centre of the tile: J_j = I / (|A| + |C_j| - I) is
// compared exactly (64-bit cross products), larger fraction then smaller
// index; with no positive J the label is 0.  Sets with more than MAXI
// items are listed for the dense path.
constexpr int JX_S = 8;
constexpr int JX_THREADS = 32 * JX_S;
// NARROW: sets of at most 128 items, 8-bit counters, tiles of 8192 centres
// (74 KB of shared memory: three blocks per SM); otherwise up to 512 items,
// 16-bit counters, tiles of 4096 centres (104 KB).
template <bool NARROW> struct Jx {
    static constexpr int KT = NARROW ? 8192 : 4096;  // centres per tile
    static constexpr int MAXI = NARROW ? 128 : 512;  // items per set on the tiled path
    static constexpr int LG = NARROW ? 2 : 1;        // log2 counters per word
    static constexpr int CBITS = 32 >> LG;
    static constexpr uint32_t CMASK = NARROW ? 0xFFu : 0xFFFFu;
    static constexpr int CW = KT >> LG;              // counter words per set
    static constexpr size_t SMEM = (size_t)JX_S * CW * 4 + (size_t)JX_S * MAXI * (4 + 4 + 2);
};

// the largest set: max over i of off[i + 1] - off[i]
__global__ void k_max_len(int64_t n, const int64_t *__restrict__ off, unsigned long long *__restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)(off[i + 1] - off[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// tile_off[r * (ntiles + 1) + t]: the first entry of posting list r whose
// centre is in tile t or later (ntiles + 1 entries per list)
__global__ void k_tile_offsets(int64_t nr, const int64_t *__restrict__ post_off,
                               const uint32_t *__restrict__ post_centre, int ntiles, int kt,
                               int32_t *__restrict__ tile_off) {
    const int64_t tot = nr * (ntiles + 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (ntiles + 1);
        const int t = (int)(e % (ntiles + 1));
        const uint64_t lim = (uint64_t)t * kt;
        int64_t lo = post_off[r], hi = post_off[r + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)post_centre[mid] < lim) lo = mid + 1;
            else hi = mid;
        }
        tile_off[e] = (int32_t)lo;
    }
}

template <bool NARROW>
__global__ void __launch_bounds__(JX_THREADS) k_jac_tiled(
    int64_t n, const int64_t *__restrict__ off, const uint32_t *__restrict__ items, int na_fix, int64_t k,
    const int32_t *__restrict__ clen, const uint64_t *__restrict__ cmask, const uint32_t *__restrict__ hv_item,
    const int16_t *__restrict__ hv_bit, int nheavy, int HW, const uint32_t *__restrict__ post_item,
    const int32_t *__restrict__ tile_off, int ntiles, int64_t n_post_items, const uint32_t *__restrict__ post_centre,
    int32_t *__restrict__ labels, int32_t *__restrict__ ovf_rows, unsigned long long *__restrict__ n_ovf) {
    using C = Jx<NARROW>;
    __shared__ unsigned long long s_am[JX_S][JX_HW];  // the sets' heavy-item masks
    extern __shared__ uint32_t jx_smem[];
    uint32_t *cnt = jx_smem;                                          // [S][KT / 2]
    int32_t *ridx = reinterpret_cast<int32_t *>(cnt + JX_S * C::CW);        // [S][MAXI]: posting list of each item
    int32_t *rps = ridx + JX_S * C::MAXI;                                  // [S][MAXI]: its range in the tile
    uint16_t *rlen = reinterpret_cast<uint16_t *>(rps + JX_S * C::MAXI);   // [S][MAXI]
    __shared__ int s_ni[JX_S];
    __shared__ int64_t s_na[JX_S];
    __shared__ uint32_t r_n[JX_S][JX_S], r_d[JX_S][JX_S];
    __shared__ int r_j[JX_S][JX_S];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < JX_S * C::CW; e += blockDim.x) cnt[e] = 0;
    const int64_t ngroups = (n + JX_S - 1) / JX_S;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        // the warp's set: posting ranges of its items
        const int64_t i = g * JX_S + w;
        int ni = 0;
        if (i < n) {
            const int64_t s0 = off[i], e0 = off[i + 1];
            ni = (int)min(e0 - s0, (int64_t)C::MAXI + 1);
            if (ni > C::MAXI) {
                if (lane == 0) ovf_rows[atomicAdd(n_ovf, 1ull)] = (int32_t)i;
                ni = 0;
            }
            if (lane < JX_HW) s_am[w][lane] = 0ull;
            __syncwarp();
            for (int p = lane; p < ni; p += 32) {
                const uint32_t it = items[s0 + p];
                const int hb = heavy_bit(it, hv_item, hv_bit, nheavy);
                if (hb >= 0) {
                    atomicOr(&s_am[w][hb >> 6], 1ull << (hb & 63));
                    ridx[w * C::MAXI + p] = -1;
                    continue;
                }
                int64_t lo = 0, hi = n_post_items;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (post_item[mid] < it) lo = mid + 1;
                    else hi = mid;
                }
                const bool f = lo < n_post_items && post_item[lo] == it;
                ridx[w * C::MAXI + p] = f ? (int32_t)lo : -1;
            }
            if (lane == 0) {
                s_ni[w] = ni;
                s_na[w] = na_fix >= 0 ? na_fix : e0 - s0;
            }
        } else if (lane == 0) {
            s_ni[w] = 0;
            s_na[w] = 0;
            for (int h = 0; h < JX_HW; h++) s_am[w][h] = 0ull;
        }
        __syncthreads();
        uint32_t bn[JX_S], bd[JX_S], na[JX_S];
        uint64_t am[JX_S][JX_HW];
        int bj[JX_S];
#pragma unroll
        for (int q = 0; q < JX_S; q++) {
            bn[q] = 0;
            bd[q] = 1;
            bj[q] = 0x7FFFFFFF;
            na[q] = (uint32_t)s_na[q];
#pragma unroll
            for (int h = 0; h < JX_HW; h++) am[q][h] = s_am[q][h];
        }
        for (int64_t c0 = 0; c0 < k; c0 += C::KT) {
            const int64_t c1 = min(k, c0 + C::KT);
            // counting: lanes walk consecutive entries of one posting list
            const int niw = s_ni[w];
            uint32_t *cw = cnt + w * C::CW;
            const int t = (int)(c0 / C::KT);
            // the items' ranges in this tile, lane per item (independent loads)
            for (int q = lane; q < niw; q += 32) {
                const int32_t r = ridx[w * C::MAXI + q];
                int32_t ps = 0, pe = 0;
                if (r >= 0) {
                    ps = tile_off[(int64_t)r * (ntiles + 1) + t];
                    pe = tile_off[(int64_t)r * (ntiles + 1) + t + 1];
                }
                rps[w * C::MAXI + q] = ps;
                rlen[w * C::MAXI + q] = (uint16_t)(pe - ps);
            }
            __syncwarp();
            // short ranges: a lane walks one item's entries
            for (int q = lane; q < niw; q += 32) {
                const int len = rlen[w * C::MAXI + q];
                if (len == 0 || len >= 32) continue;
                const int32_t ps = rps[w * C::MAXI + q];
                for (int e = 0; e < len; e++) {
                    const int cc = (int)((int64_t)post_centre[ps + e] - c0);
                    atomicAdd(&cw[cc >> C::LG], 1u << ((cc & ((1 << C::LG) - 1)) * C::CBITS));
                }
            }
            // long ranges: the warp walks one item's entries, lane per entry
            for (int q = 0; q < niw; q++) {
                const int len = rlen[w * C::MAXI + q];
                if (len < 32) continue;
                const int32_t ps = rps[w * C::MAXI + q];
#pragma unroll 4
                for (int p = lane; p < len; p += 32) {
                    const int cc = (int)((int64_t)post_centre[ps + p] - c0);
                    atomicAdd(&cw[cc >> C::LG], 1u << ((cc & ((1 << C::LG) - 1)) * C::CBITS));
                }
            }
            __syncwarp();
            __syncthreads();
            // scoring: thread per centre of the tile, all JX_S sets
            for (int cc = threadIdx.x; cc < (int)(c1 - c0); cc += blockDim.x) {
                const int64_t c = c0 + cc;
                const int64_t cl = clen[c];
                uint64_t cm[JX_HW];
#pragma unroll
                for (int h = 0; h < JX_HW; h++) cm[h] = h < HW ? cmask[c * HW + h] : 0ull;
#pragma unroll
                for (int q = 0; q < JX_S; q++) {
                    uint32_t in = (cnt[q * C::CW + (cc >> C::LG)] >> ((cc & ((1 << C::LG) - 1)) * C::CBITS)) & C::CMASK;
#pragma unroll
                    for (int h = 0; h < JX_HW; h++) in += __popcll(am[q][h] & cm[h]);
                    if (in) {
                        // |A| + |C| < 2^16: both cross products fit 32 bits
                        const uint32_t un = na[q] + (uint32_t)cl - in;
                        const uint32_t l = in * bd[q], r = bn[q] * un;
                        if (l > r || (l == r && (int)c < bj[q])) {
                            bn[q] = in;
                            bd[q] = un;
                            bj[q] = (int)c;
                        }
                    }
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < JX_S * C::CW; e += blockDim.x) cnt[e] = 0;
            __syncthreads();
        }
        // per set: reduce the threads' bests (warp, then across warps)
#pragma unroll
        for (int q = 0; q < JX_S; q++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint32_t on = __shfl_xor_sync(0xffffffffu, bn[q], o);
                const uint32_t od = __shfl_xor_sync(0xffffffffu, bd[q], o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj[q], o);
                const uint32_t l = on * bd[q], r = bn[q] * od;
                if (l > r || (l == r && oj < bj[q])) {
                    bn[q] = on;
                    bd[q] = od;
                    bj[q] = oj;
                }
            }
            if (lane == 0) {
                r_n[q][w] = bn[q];
                r_d[q][w] = bd[q];
                r_j[q][w] = bj[q];
            }
        }
        __syncthreads();
        if (threadIdx.x < JX_S) {
            const int q = threadIdx.x;
            uint32_t n0 = 0, d0 = 1;
            int j0 = 0x7FFFFFFF;
            for (int v = 0; v < JX_S; v++) {
                const uint32_t l = r_n[q][v] * d0, r = n0 * r_d[q][v];
                if (l > r || (l == r && r_j[q][v] < j0)) {
                    n0 = r_n[q][v];
                    d0 = r_d[q][v];
                    j0 = r_j[q][v];
                }
            }
            const int64_t ii = g * JX_S + q;
            // no positive J: every fraction is 0 and the smallest index wins
            if (ii < n) labels[ii] = (n0 > 0 && j0 != 0x7FFFFFFF) ? j0 : 0;
        }
        __syncthreads();
    }
}

}  // namespace

// Majority set of each group of sets: items present in more than half of
// the group's member sets (groups CSR goff/gmem of set indices; sets CSR
// soff/sids).  Output CSR has one (possibly empty) entry per group.
geek_status majority_per_group(geek_ctx *ctx, Scratch &scr, int64_t ng, const int64_t *goff, const int32_t *gmem,
                               int64_t m, const int64_t *soff, const uint32_t *sids, int64_t **out_off,
                               uint32_t **out_ids, int64_t *out_n, cudaStream_t st) {
    int64_t *w, *woff, *T_dev, *cnt, *coff, *tot;
    int32_t *gid;
    GK_TRY(scr.alloc(&w, std::max<int64_t>(m, 1)));
    GK_TRY(scr.alloc(&woff, std::max<int64_t>(m, 1)));
    GK_TRY(scr.alloc(&gid, std::max<int64_t>(m, 1)));
    GK_TRY(scr.alloc(&T_dev, 1));
    GK_TRY(scr.alloc(&cnt, ng));
    GK_TRY(scr.alloc(out_off, ng + 1));
    GK_TRY(scr.alloc(&tot, 1));
    GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * ng, st));
    GK_COUNT();
    k_group_w<<<G(ctx, m), 256, 0, st>>>(m, gmem, soff, w);
    GK_COUNT();
    k_group_of<<<G(ctx, ng), 256, 0, st>>>(ng, goff, gid);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, w, woff, m, T_dev, st));
    int64_t T = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&T, T_dev, 8, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t total = 0;
    if (T > 0) {
        uint64_t *pairs;
        GK_TRY(scr.alloc(&pairs, T));
        GK_COUNT();
        k_group_expand<<<G(ctx, m), 256, 0, st>>>(m, gid, gmem, woff, soff, sids, pairs);
        GK_LAUNCH(ctx);
        GK_TRY(radix_sort_segments(ctx, scr, 1, T, &pairs, nullptr, nullptr, 32 + bit_length_u64((uint64_t)ng), st));
        int64_t *prs, *nr;
        GK_TRY(scr.alloc(&prs, T + 1));
        GK_TRY(scr.alloc(&nr, 1));
        GK_TRY(segment_runs(ctx, scr, 1, T, pairs, nullptr, nullptr, prs, nr, st));
        int64_t NR = 0;
        GK_CUDA(ctx, cudaMemcpyAsync(&NR, nr, 8, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        int64_t *keep, *pos, *ktot;
        GK_TRY(scr.alloc(&keep, NR));
        GK_TRY(scr.alloc(&pos, NR));
        GK_TRY(scr.alloc(&ktot, 1));
        GK_COUNT();
        k_group_keep<<<G(ctx, NR), 256, 0, st>>>(nr, prs, pairs, goff, keep, cnt);
        GK_LAUNCH(ctx);
        GK_TRY(exclusive_scan_i64(ctx, scr, keep, pos, NR, ktot, st));
        GK_CUDA(ctx, cudaMemcpyAsync(&total, ktot, 8, cudaMemcpyDeviceToHost, st));
        GK_TRY(sort_err_check(ctx, st));  // synchronises st
        GK_TRY(scr.alloc(out_ids, std::max<int64_t>(1, total)));
        GK_COUNT();
        k_group_emit<<<G(ctx, NR), 256, 0, st>>>(nr, prs, pairs, keep, pos, *out_ids);
        GK_LAUNCH(ctx);
    } else {
        GK_TRY(scr.alloc(out_ids, 1));
    }
    GK_TRY(exclusive_scan_i64(ctx, scr, cnt, *out_off, ng, tot, st));
    GK_CUDA(ctx, cudaMemcpyAsync(*out_off + ng, tot, 8, cudaMemcpyDeviceToDevice, st));
    *out_n = total;
    (void)coff;
    return GEEK_OK;
}

geek_status assign_hetero(geek_ctx *ctx, Scratch &scr, const geek_buckets *b, const uint32_t *tok, int n_cat,
                          const silk_seeds *s, int32_t *labels, geek_assign_stats *stats, geek_centres *keep,
                          cudaStream_t st) {
    const int64_t n = b->n, k = s->k;
    const int A = b->L + n_cat;
    if (stats) *stats = geek_assign_stats{0.0, 0.0, k, 0};
    if (A > CAT_MAXA) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than %d categorical attributes", CAT_MAXA);
    if (n == 0) return GEEK_OK;
    uint64_t *attrs, *modes;
    int32_t *matches;
    GK_TRY(scr.alloc(&attrs, (size_t)n * A));
    GK_TRY(scr.alloc(&modes, (size_t)std::max<int64_t>(k, 1) * A));
    GK_TRY(scr.alloc(&matches, n));
    int32_t *rep = nullptr;
    if (keep && k) GK_TRY(scr.alloc(&rep, (size_t)k * A));
    GK_COUNT();
    k_build_attrs<<<G(ctx, n * A), 256, 0, st>>>(n, b->L, n_cat, b->num_key, tok, attrs);
    if (k) GK_COUNT(), k_modes<<<G(ctx, k * A), 256, 0, st>>>(k, A, s->off, s->ids, attrs, modes, rep);
    GK_LAUNCH(ctx);
    if (keep) {
        keep->kind = GEEK_HETERO;
        keep->k = k;
        keep->n_attr = A;
        GK_TRY(own_alloc(ctx, (void **)&keep->modes, sizeof(int64_t) * (size_t)std::max<int64_t>(k, 1) * A, st));
        if (k) {
            int64_t *flags, *excl, *tbase;
            GK_TRY(scr.alloc(&flags, std::max<int64_t>(b->NB, 1)));
            GK_TRY(scr.alloc(&excl, std::max<int64_t>(b->NB, 1)));
            GK_TRY(scr.alloc(&tbase, b->L));
            std::vector<int64_t> hb(b->L, 0);
            for (int l = 1; l < b->L; l++) hb[l] = hb[l - 1] + b->nb[l - 1];
            GK_CUDA(ctx, cudaMemcpyAsync(tbase, hb.data(), sizeof(int64_t) * b->L, cudaMemcpyHostToDevice, st));
            for (int l = 0; l < b->L; l++) {
                GK_COUNT();
                k_num_run_flags<<<G(ctx, b->nb[l]), 256, 0, st>>>(b->nb[l], hb[l], b->boff, b->members,
                                                                 b->num_key + (int64_t)l * n, flags);
            }
            GK_LAUNCH(ctx);
            GK_TRY(exclusive_scan_i64(ctx, scr, flags, excl, b->NB, nullptr, st));
            GK_COUNT();
            k_mode_out<<<G(ctx, k * A), 256, 0, st>>>(k, A, b->L, n, modes, rep, b->obj_bucket, tbase, excl, flags,
                                                      keep->modes);
            GK_LAUNCH(ctx);
            // the host vector hb must outlive the copy above
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
    }
    GK_COUNT();
    k_assign_cat<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, A, k, attrs, modes, labels, matches);
    GK_LAUNCH(ctx);
    if (stats) {
        // SSE in the categorical distance 1 - m / (2A - m), computed on the host
        std::vector<int32_t> hm(n);
        GK_CUDA(ctx, cudaMemcpyAsync(hm.data(), matches, 4 * n, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        double sse = 0.0, rmax = 0.0;
        for (int64_t i = 0; i < n; i++) {
            if (hm[i] < 0) continue;
            const double dd = 1.0 - (double)hm[i] / (double)(2 * A - hm[i]);
            sse += dd;
            rmax = std::max(rmax, dd);
        }
        stats->sse = sse;
        stats->radius_max = rmax;
    }
    return GEEK_OK;
}

geek_status jaccard_core(geek_ctx *ctx, Scratch &scr, const int64_t *off, const uint32_t *items, int64_t n,
                         int na_fix, int64_t k, const int64_t *coff, const uint32_t *citems, int64_t nci,
                         int32_t *labels, geek_assign_stats *stats, cudaStream_t st);

geek_status assign_sets(geek_ctx *ctx, Scratch &scr, const int64_t *off, const uint32_t *items, int64_t n,
                        const silk_seeds *s, int32_t *labels, geek_assign_stats *stats, geek_centres *keep,
                        cudaStream_t st) {
    const int64_t k = s->k;
    if (stats) *stats = geek_assign_stats{0.0, 0.0, k, 0};
    if (keep) {
        keep->kind = GEEK_SETS;
        keep->k = k;
    }
    if (n == 0 || k == 0) {
        if (keep) {
            GK_TRY(own_alloc(ctx, (void **)&keep->item_off, sizeof(int64_t) * (size_t)(k + 1), st));
            GK_CUDA(ctx, cudaMemsetAsync(keep->item_off, 0, sizeof(int64_t) * (size_t)(k + 1), st));
        }
        if (n && k == 0) GK_CUDA(ctx, cudaMemsetAsync(labels, 0xFF, sizeof(int32_t) * n, st));
        return GEEK_OK;
    }
    // centres: majority item sets of the seeds
    int64_t *coff, nci = 0;
    uint32_t *citems;
    GK_TRY(majority_per_group(ctx, scr, k, s->off, s->ids, s->n_ids, off, items, &coff, &citems, &nci, st));
    if (keep) {
        keep->n_items = nci;
        GK_TRY(own_alloc(ctx, (void **)&keep->item_off, sizeof(int64_t) * (size_t)(k + 1), st));
        GK_TRY(own_alloc(ctx, (void **)&keep->items, sizeof(uint32_t) * (size_t)std::max<int64_t>(nci, 1), st));
        GK_CUDA(ctx, cudaMemcpyAsync(keep->item_off, coff, sizeof(int64_t) * (size_t)(k + 1), cudaMemcpyDeviceToDevice, st));
        if (nci)
            GK_CUDA(ctx, cudaMemcpyAsync(keep->items, citems, sizeof(uint32_t) * (size_t)nci, cudaMemcpyDeviceToDevice, st));
    }
    return jaccard_core(ctx, scr, off, items, n, -1, k, coff, citems, nci, labels, stats, st);
}

// Exact Jaccard argmax of every set against k centre sets (CSR coff /
// citems, nci items): J_j = |A n C_j| / |A u C_j|, larger fraction then
// smaller index; with no positive J the label is 0.  na_fix >= 0 gives every
// set the size na_fix (rows padded with an id that no centre holds).
geek_status jaccard_core(geek_ctx *ctx, Scratch &scr, const int64_t *off, const uint32_t *items, int64_t n,
                         int na_fix, int64_t k, const int64_t *coff, const uint32_t *citems, int64_t nci,
                         int32_t *labels, geek_assign_stats *stats, cudaStream_t st) {
    // inverted index item -> centres: pairs sorted by (item, centre), runs of
    // equal items, one posting list (ascending centres) per distinct item
    uint64_t *pairs, *ikey;
    GK_TRY(scr.alloc(&pairs, std::max<int64_t>(nci, 1)));
    GK_TRY(scr.alloc(&ikey, std::max<int64_t>(nci, 1)));
    GK_COUNT();
    k_centre_pairs<<<G(ctx, k), 256, 0, st>>>(k, coff, citems, pairs);
    GK_LAUNCH(ctx);
    GK_TRY(radix_sort_segments(ctx, scr, 1, nci, &pairs, nullptr, nullptr, 64, st));
    GK_COUNT();
    k_item_key<<<G(ctx, nci), 256, 0, st>>>(nci, pairs, ikey);
    GK_LAUNCH(ctx);
    int64_t *rs, *nr_dev;
    GK_TRY(scr.alloc(&rs, nci + 1));
    GK_TRY(scr.alloc(&nr_dev, 1));
    GK_TRY(segment_runs(ctx, scr, 1, nci, ikey, nullptr, nullptr, rs, nr_dev, st));
    int64_t ni = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&ni, nr_dev, 8, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    // heavy items: the (up to 64 JX_HW) longest posting lists of length >= 2,
    // chosen on the host from the run lengths; the others keep posting lists
    std::vector<int64_t> hrs(ni + 1);
    GK_CUDA(ctx, cudaMemcpyAsync(hrs.data(), rs, 8 * (ni + 1), cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> ord(ni);
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    for (int64_t r = 0; r < ni; r++) ord[r] = (int32_t)r;
    const int64_t hmax = std::min<int64_t>(64 * JX_HW, ni);
    std::partial_sort(ord.begin(), ord.begin() + hmax, ord.end(), [&](int32_t a, int32_t b) {
        const int64_t la = hrs[a + 1] - hrs[a], lb = hrs[b + 1] - hrs[b];
        return la != lb ? la > lb : a < b;
    });
    int nheavy = 0;
    while (nheavy < hmax && hrs[ord[nheavy] + 1] - hrs[ord[nheavy]] >= 2) nheavy++;
    const int HW = (nheavy + 63) / 64;
    std::vector<int64_t> h_is(ni, 0);
    std::vector<int32_t> hv_runs(ord.begin(), ord.begin() + nheavy);
    std::sort(hv_runs.begin(), hv_runs.end());  // runs ascend with the item value
    std::vector<int16_t> h_bit(nheavy);
    std::vector<int32_t> rank_of(ni, -1);
    for (int b = 0; b < nheavy; b++) rank_of[ord[b]] = b;  // bit = rank by posting length
    for (int q = 0; q < nheavy; q++) {
        h_is[hv_runs[q]] = 1;
        h_bit[q] = (int16_t)rank_of[hv_runs[q]];
    }
    uint32_t *d_litem, *d_lcentre, *hv_item;
    int16_t *hv_bit;
    int64_t *is_heavy, *lrun, *lrun_pos, *lent, *lent_pos, *d_loff, *nlight, *nlent, *hv_run_dev;
    GK_TRY(scr.alloc(&is_heavy, std::max<int64_t>(ni, 1)));
    GK_TRY(scr.alloc(&hv_item, std::max(1, nheavy)));
    GK_TRY(scr.alloc(&hv_bit, std::max(1, nheavy)));
    GK_TRY(scr.alloc(&hv_run_dev, std::max(1, nheavy)));
    GK_TRY(scr.alloc(&lrun, std::max<int64_t>(ni, 1)));
    GK_TRY(scr.alloc(&lrun_pos, std::max<int64_t>(ni, 1)));
    GK_TRY(scr.alloc(&lent, std::max<int64_t>(ni, 1)));
    GK_TRY(scr.alloc(&lent_pos, std::max<int64_t>(ni, 1)));
    GK_TRY(scr.alloc(&nlight, 1));
    GK_TRY(scr.alloc(&nlent, 1));
    GK_CUDA(ctx, cudaMemcpyAsync(is_heavy, h_is.data(), 8 * ni, cudaMemcpyHostToDevice, st));
    if (nheavy) {
        std::vector<int64_t> hv_r64(hv_runs.begin(), hv_runs.end());
        GK_CUDA(ctx, cudaMemcpyAsync(hv_run_dev, hv_r64.data(), 8 * nheavy, cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaMemcpyAsync(hv_bit, h_bit.data(), 2 * nheavy, cudaMemcpyHostToDevice, st));
        GK_COUNT();
        k_run_items<<<G(ctx, nheavy), 256, 0, st>>>(nheavy, hv_run_dev, rs, ikey, hv_item);
        GK_LAUNCH(ctx);
    }
    // the host vectors above must outlive their copies
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    GK_COUNT();
    k_light_flags<<<G(ctx, ni), 256, 0, st>>>(ni, rs, is_heavy, lrun, lent);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, lrun, lrun_pos, ni, nlight, st));
    GK_TRY(exclusive_scan_i64(ctx, scr, lent, lent_pos, ni, nlent, st));
    int64_t h_nlight = 0, h_nlent = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_nlight, nlight, 8, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaMemcpyAsync(&h_nlent, nlent, 8, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    GK_TRY(scr.alloc(&d_litem, std::max<int64_t>(1, h_nlight)));
    GK_TRY(scr.alloc(&d_loff, h_nlight + 1));
    GK_TRY(scr.alloc(&d_lcentre, std::max<int64_t>(1, h_nlent)));
    GK_COUNT();
    k_light_emit<<<G(ctx, ni), 256, 0, st>>>(ni, rs, ikey, pairs, is_heavy, lrun_pos, lent_pos, d_litem, d_loff,
                                             d_lcentre, nlent, h_nlight);
    GK_LAUNCH(ctx);
    uint64_t *cmask;
    int32_t *clen, *counts;
    GK_TRY(scr.alloc(&cmask, (size_t)k * std::max(HW, 1)));
    GK_TRY(scr.alloc(&clen, k));
    GK_COUNT();
    k_heavy_masks<<<G(ctx, k), 256, 0, st>>>(k, coff, citems, hv_item, hv_bit, nheavy, HW, cmask, clen);
    GK_LAUNCH(ctx);
    if (nci > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 2^31 centre items");
    // the tiled kernel compares fractions in 32 bits: |A| <= MAXI (else the
    // dense path) and every |C| below 2^15; the narrow variant when no set has
    // more than its MAXI items
    bool tiled_ok = na_fix < 32768;
    unsigned long long h_amax = 0, *d_amax;
    GK_TRY(scr.alloc(&d_amax, 1));
    GK_CUDA(ctx, cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long), st));
    if (na_fix < 0 && n > 0) {
        GK_COUNT();
        k_max_len<<<G(ctx, n), 256, 0, st>>>(n, off, d_amax);
        GK_LAUNCH(ctx);
    }
    {
        std::vector<int64_t> hco(k + 1);
        GK_CUDA(ctx, cudaMemcpyAsync(hco.data(), coff, 8 * (k + 1), cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaMemcpyAsync(&h_amax, d_amax, sizeof h_amax, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        for (int64_t j = 0; j < k && tiled_ok; j++) tiled_ok = hco[j + 1] - hco[j] < 32768;
    }
    const bool narrow = (na_fix >= 0 ? (int64_t)na_fix : (int64_t)h_amax) <= Jx<true>::MAXI;
    int32_t *ovf;
    unsigned long long *n_ovf;
    GK_TRY(scr.alloc(&ovf, n));
    GK_TRY(scr.alloc(&n_ovf, 1));
    GK_CUDA(ctx, cudaMemsetAsync(n_ovf, 0, sizeof(unsigned long long), st));
    {
        static bool attr = false;
        if (!attr) {
            GK_CUDA(ctx, cudaFuncSetAttribute(k_jac_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)Jx<true>::SMEM));
            GK_CUDA(ctx, cudaFuncSetAttribute(k_jac_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)Jx<false>::SMEM));
            attr = true;
        }
        const int kt = narrow ? Jx<true>::KT : Jx<false>::KT;
        const int ntiles = (int)ceil_div(k, kt);
        int32_t *toff;
        GK_TRY(scr.alloc(&toff, (size_t)std::max<int64_t>(h_nlight, 1) * (ntiles + 1)));
        GK_COUNT();
        k_tile_offsets<<<G(ctx, h_nlight * (ntiles + 1)), 256, 0, st>>>(h_nlight, d_loff, d_lcentre, ntiles, kt, toff);
        EvTimer tk(ctx, "kernel.jaccard", st);
        tk.work = (double)n * (double)k;  // (set, centre) pairs scored
        if (!tiled_ok) {  // very large central sets: every set takes the dense path
            GK_COUNT();
            k_iota_rows<<<G(ctx, n), 256, 0, st>>>(n, ovf, n_ovf);
            GK_LAUNCH(ctx);
        } else {
        GK_COUNT();
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, JX_S), (int64_t)ctx->num_sms * 3);
        if (narrow)
            k_jac_tiled<true><<<grid, JX_THREADS, Jx<true>::SMEM, st>>>(n, off, items, na_fix, k, clen, cmask, hv_item,
                                                                      hv_bit, nheavy, HW, d_litem, toff, ntiles,
                                                                      h_nlight, d_lcentre, labels, ovf, n_ovf);
        else
            k_jac_tiled<false><<<grid, JX_THREADS, Jx<false>::SMEM, st>>>(n, off, items, na_fix, k, clen, cmask,
                                                                        hv_item, hv_bit, nheavy, HW, d_litem, toff,
                                                                        ntiles, h_nlight, d_lcentre, labels, ovf,
                                                                        n_ovf);
        GK_LAUNCH(ctx);
        }
    }
    unsigned long long h_ovf = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_ovf, n_ovf, sizeof h_ovf, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_ovf) {
        // sets with too many light candidates: every centre scanned per set
        const int blocks = (int)std::min<int64_t>(ctx->num_sms * 4, ceil_div((int64_t)h_ovf, 8));
        const int64_t nwarps = (int64_t)blocks * 8;
        GK_TRY(scr.alloc(&counts, (size_t)nwarps * k));
        GK_CUDA(ctx, cudaMemsetAsync(counts, 0, sizeof(int32_t) * nwarps * k, st));
        GK_COUNT();
        k_assign_jaccard<<<blocks, 256, 0, st>>>(n, off, items, k, clen, cmask, hv_item, hv_bit, nheavy, HW, d_litem,
                                                 d_loff, h_nlight, d_lcentre, counts, labels, ovf, n_ovf, na_fix);
        GK_LAUNCH(ctx);
    }
    if (stats) stats->n_recheck_rows = (int64_t)h_ovf;  // sets decided by the dense path
    return sort_err_check(ctx, st);  // synchronises st
}

namespace {

// id of each token in the sorted distinct list U (nu entries), or 2^32 - 1
// when absent (no centre holds it)
__global__ void k_map_tokens(int64_t m, const uint64_t *__restrict__ tok, const uint64_t *__restrict__ U, int64_t nu,
                             uint32_t *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = tok[e];
        int64_t lo = 0, hi = nu;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (U[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        out[e] = (lo < nu && U[lo] == v) ? (uint32_t)lo : 0xFFFFFFFFu;
    }
}

__global__ void k_fixed_off(int64_t n, int64_t len, int64_t *__restrict__ off) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        off[i] = i * len;
}

// the first token of each run of equal sorted tokens: compacted to U
__global__ void k_run_firsts(int64_t m, const uint64_t *__restrict__ sorted, const int64_t *__restrict__ rank_excl,
                             uint64_t *__restrict__ U) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        if (e == 0 || sorted[e] != sorted[e - 1]) U[rank_excl[e]] = sorted[e];
}

__global__ void k_run_flags(int64_t m, const uint64_t *__restrict__ sorted, int64_t *__restrict__ flags) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        flags[e] = (e == 0 || sorted[e] != sorted[e - 1]) ? 1 : 0;
}

}  // namespace

// Sparse sets reduced by DOPH (Alg. 3): every object is its D' tokens, one per
// reduced dimension.  Central vector = the mode of each dimension over the
// seed's members (Sect. 3.3: the mode of sparse data after DOPH; ties to the
// smallest token); distance 1 - Jaccard of the token sets, i.e. the label
// maximises the number of dimensions equal to the centre's mode.  Tokens map
// to 32-bit ids of the distinct mode tokens and the Jaccard engine decides,
// with |A| = |C| = D'.
geek_status assign_doph(geek_ctx *ctx, Scratch &scr, const geek_buckets *b, const silk_seeds *s, int32_t *labels,
                        geek_assign_stats *stats, geek_centres *keep, cudaStream_t st) {
    const int64_t n = b->n, k = s->k;
    const int D = b->doph_bins;
    if (stats) *stats = geek_assign_stats{0.0, 0.0, k, 0};
    if (keep) {
        keep->kind = GEEK_SETS;
        keep->k = k;
        keep->n_attr = D;
        GK_TRY(own_alloc(ctx, (void **)&keep->modes, sizeof(int64_t) * (size_t)std::max<int64_t>(k, 1) * D, st));
    }
    if (n == 0) return GEEK_OK;
    if (k == 0) {
        GK_CUDA(ctx, cudaMemsetAsync(labels, 0xFF, sizeof(int32_t) * n, st));
        return GEEK_OK;
    }
    const int64_t km = k * D;
    uint64_t *modes, *srt;
    GK_TRY(scr.alloc(&modes, km));
    GK_TRY(scr.alloc(&srt, km));
    GK_COUNT();
    k_modes<<<G(ctx, km), 256, 0, st>>>(k, D, s->off, s->ids, b->doph_tok, modes, nullptr);
    GK_LAUNCH(ctx);
    if (keep) GK_CUDA(ctx, cudaMemcpyAsync(keep->modes, modes, 8 * km, cudaMemcpyDeviceToDevice, st));
    // distinct mode tokens, ascending
    GK_CUDA(ctx, cudaMemcpyAsync(srt, modes, 8 * km, cudaMemcpyDeviceToDevice, st));
    GK_TRY(radix_sort_segments(ctx, scr, 1, km, &srt, nullptr, nullptr, 64, st));
    int64_t *flags, *rexcl, *nu_dev;
    GK_TRY(scr.alloc(&flags, km));
    GK_TRY(scr.alloc(&rexcl, km));
    GK_TRY(scr.alloc(&nu_dev, 1));
    GK_COUNT();
    k_run_flags<<<G(ctx, km), 256, 0, st>>>(km, srt, flags);
    GK_LAUNCH(ctx);
    GK_TRY(exclusive_scan_i64(ctx, scr, flags, rexcl, km, nu_dev, st));
    int64_t nu = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&nu, nu_dev, 8, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    if (nu >= 0xFFFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "too many distinct mode tokens");
    uint64_t *U;
    GK_TRY(scr.alloc(&U, nu));
    GK_COUNT();
    k_run_firsts<<<G(ctx, km), 256, 0, st>>>(km, srt, rexcl, U);
    // centres and rows as id lists of fixed length D
    uint32_t *cid, *rid;
    int64_t *coff, *roff;
    GK_TRY(scr.alloc(&cid, km));
    GK_TRY(scr.alloc(&rid, n * D));
    GK_TRY(scr.alloc(&coff, k + 1));
    GK_TRY(scr.alloc(&roff, n + 1));
    GK_COUNT();
    k_map_tokens<<<G(ctx, km), 256, 0, st>>>(km, modes, U, nu, cid);
    GK_COUNT();
    k_map_tokens<<<G(ctx, n * D), 256, 0, st>>>(n * D, b->doph_tok, U, nu, rid);
    GK_COUNT();
    k_fixed_off<<<G(ctx, k + 1), 256, 0, st>>>(k, D, coff);
    GK_COUNT();
    k_fixed_off<<<G(ctx, n + 1), 256, 0, st>>>(n, D, roff);
    GK_LAUNCH(ctx);
    return jaccard_core(ctx, scr, roff, rid, n, D, k, coff, cid, km, labels, stats, st);
}
