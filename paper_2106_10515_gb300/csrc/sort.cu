// Device radix sort, run detection and prefix sums: the grouping machinery
// behind bucket formation (T[G(x)].push(j) in Algs. 2-3), SILK bins (Alg. 4)
// and majority voting.  Sorting is a stable LSD radix sort with 8-bit digits
// over S equal-length segments at once (one segment per hash table), so the
// L tables of a transform share every launch; each pass is one kernel whose
// tiles find their output offsets by decoupled look-back.
#include <cstdarg>

#include "common.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 10;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 2560 elements per tile
constexpr int NWARP = RS_THREADS / 32;

// ---- block-wide exclusive scan helper (uint32, 1024 threads max) ----------
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total, uint32_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) wsum[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t before = warp ? wsum[warp - 1] : 0;
    *total = wsum[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// exclusive scan in place of each segment's `len` counters; optional total
__global__ void __launch_bounds__(1024) k_seg_scan_u32(uint32_t *__restrict__ c, int64_t len,
                                                       int64_t *__restrict__ totals) {
    __shared__ uint32_t wsum[32];
    uint32_t *a = c + (int64_t)blockIdx.x * len;
    uint32_t carry = 0;
    for (int64_t base = 0; base < len; base += 1024 * 4) {
        int64_t p0 = base + (int64_t)threadIdx.x * 4;
        uint32_t v[4], s = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[k] = p0 + k < len ? a[p0 + k] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_excl_scan<1024>(s, &tot, wsum) + carry;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (p0 + k < len) a[p0 + k] = ex;
            ex += v[k];
        }
        carry += tot;
    }
    if (totals && threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// ---- one-sweep passes (decoupled look-back) --------------------------------
// Digit totals do not change from one LSD pass to the next (a pass only
// permutes a segment), so one read of the keys gives every pass its global
// digit offsets.  Each pass is then a single kernel: a block takes the next
// tile of its segment in launch order (a global ticket), publishes the
// tile's per-digit count, and adds up its predecessors' counts by looking
// back through their published words until one carries an inclusive prefix.
// Word layout: bits 31..30 = state (0 empty, 1 tile count, 2 inclusive
// prefix), bits 29..0 = count; segments are limited to 2^30 - 1 elements.
constexpr uint32_t LB_AGG = 1u << 30, LB_PREFIX = 2u << 30, LB_MASK = (1u << 30) - 1;
constexpr int HIST_BLOCKS_PER_SEG = 96;

__device__ __forceinline__ unsigned long long sort_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// counts[seg][pass][256] += digit counts of every pass (counts zeroed first).
// Shared histograms per warp pair keep same-address atomics rare when a
// high digit takes few values.
__global__ void __launch_bounds__(256) k_rs_hist_all(const uint64_t *__restrict__ lo, const uint64_t *__restrict__ hi,
                                                     int64_t m, int npass, uint32_t *__restrict__ counts) {
    extern __shared__ uint32_t hs[];  // [4][npass][256]
    const int seg = blockIdx.y, t = threadIdx.x, sub = (t >> 6);
    for (int i = t; i < 4 * npass * 256; i += 256) hs[i] = 0;
    __syncthreads();
    const uint64_t *l = lo + (int64_t)seg * m;
    const uint64_t *h = hi ? hi + (int64_t)seg * m : nullptr;
    uint32_t *my = hs + sub * npass * 256;
    for (int64_t p = (int64_t)blockIdx.x * 256 + t; p < m; p += (int64_t)gridDim.x * 256) {
        const uint64_t kl = l[p];
        const uint64_t kh = h ? h[p] : 0;
        for (int q = 0; q < npass; q++) {
            const int sh = q * 8;
            const uint32_t d = (uint32_t)(((sh >= 64 ? kh : kl) >> (sh & 63)) & 0xFFu);
            atomicAdd(&my[q * 256 + d], 1u);
        }
    }
    __syncthreads();
    for (int i = t; i < npass * 256; i += 256) {
        const uint32_t c = hs[i] + hs[npass * 256 + i] + hs[2 * npass * 256 + i] + hs[3 * npass * 256 + i];
        if (c) atomicAdd(&counts[(int64_t)seg * npass * 256 + i], c);
    }
}

// exclusive scan of every (segment, pass) row of 256 digit counts, in place
__global__ void __launch_bounds__(256) k_rs_base_all(uint32_t *__restrict__ counts) {
    __shared__ uint32_t wsum[32];
    uint32_t *a = counts + (int64_t)blockIdx.x * 256;
    const uint32_t v = a[threadIdx.x];
    uint32_t tot;
    a[threadIdx.x] = block_excl_scan<256>(v, &tot, wsum);
}

// One pass.  A tile of RS_TILE elements is split into 8 warp slices; warp w
// reads its slice striped (item i of lane l is element w*IT*32 + i*32 + l),
// so (warp, item, lane) is input order.  Each warp ranks its elements per
// digit with match-any, the block turns per-warp counts into tile offsets,
// stages the tile in shared memory in (digit, input order) and writes it out
// contiguously per digit: coalesced, stable.  Small tiles and 4 blocks per
// SM: the pass is latency bound, and occupancy pays more than long tiles.
template <bool HI, bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 4)
    k_rs_onesweep(const uint64_t *__restrict__ lo_in, const uint64_t *__restrict__ hi_in,
                  const uint32_t *__restrict__ v_in, uint64_t *__restrict__ lo_out,
                  uint64_t *__restrict__ hi_out, uint32_t *__restrict__ v_out, int64_t m, int tiles,
                  int dsel, int sh, const uint32_t *__restrict__ dbase, int dstride, uint32_t *__restrict__ look,
                  uint32_t *__restrict__ ticket, int *__restrict__ err, unsigned long long wait_ns,
                  int stall_tile) {
    __shared__ uint32_t whist[NWARP][256];
    __shared__ uint32_t tstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_idx;
    extern __shared__ uint64_t stage[];
    uint64_t *st_lo = stage;
    uint64_t *st_hi = stage + RS_TILE;
    uint32_t *st_v = (uint32_t *)(stage + (HI ? 2 : 1) * RS_TILE);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) s_idx = atomicAdd(ticket, 1u);
#pragma unroll
    for (int w = 0; w < NWARP; w++) whist[w][t] = 0;
    __syncthreads();
    const uint32_t idx = s_idx;
    // tickets interleave the segments: a tile's predecessor in its own
    // segment took its ticket S tickets earlier
    const int S = (int)(gridDim.x / (uint32_t)tiles);
    const int seg = (int)(idx % (uint32_t)S), tile = (int)(idx / (uint32_t)S);
    const int64_t so = (int64_t)seg * m;
    const int64_t t0 = (int64_t)tile * RS_TILE;
    const uint32_t lt = (1u << lane) - 1;
    constexpr int IT = RS_TILE / RS_THREADS;
    uint64_t klo[IT], khi[IT];
    uint32_t vv[IT], dr[IT];
    // every load of the tile in flight before the first (synchronising) rank step
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int64_t p = t0 + warp * (IT * 32) + i * 32 + lane;
        const bool valid = p < m;
        klo[i] = valid ? lo_in[so + p] : 0;
        khi[i] = (HI && valid) ? hi_in[so + p] : 0;
        vv[i] = (VALS && valid) ? v_in[so + p] : 0;
    }
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const bool valid = t0 + warp * (IT * 32) + i * 32 + lane < m;
        const uint32_t d = valid ? (uint32_t)(((dsel ? khi[i] : klo[i]) >> sh) & 0xFFu) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d < 256) {
            old = whist[warp][d];
            whist[warp][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        dr[i] = d | ((old + __popc(peers & lt)) << 9);
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NWARP; w++) {
        const uint32_t c = whist[w][t];
        whist[w][t] = run;
        run += c;
    }
    // publish this tile's count of digit t; the look-back comes after the
    // tile is staged, so that predecessors have had time to finish theirs
    uint32_t *lk = look + (int64_t)seg * tiles * 256;
    volatile uint32_t *vlk = lk;
    if (tile != stall_tile) vlk[(int64_t)tile * 256 + t] = (tile == 0 ? LB_PREFIX : LB_AGG) | run;
    uint32_t tot;
    tstart[t] = block_excl_scan<RS_THREADS>(run, &tot, wsum);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const uint32_t d = dr[i] & 511u;
        if (d < 256) {
            const uint32_t lp = tstart[d] + whist[warp][d] + (dr[i] >> 9);
            st_lo[lp] = klo[i];
            if (HI) st_hi[lp] = khi[i];
            if (VALS) st_v[lp] = vv[i];
        }
    }
    // look back over the predecessors of this segment, four words per read
    uint32_t excl = 0;
    bool gave_up = false;
    if (tile > 0) {
        int j = tile - 1;
        unsigned long long w0 = 0;
        for (uint32_t it = 0;; it++) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; k++) w[k] = j - k >= 0 ? vlk[(int64_t)(j - k) * 256 + t] : 0u;
            int k = 0;
            bool done = false;
            for (; k < 4; k++) {
                const uint32_t stt = w[k] & ~LB_MASK;
                if (stt == 0) break;  // not published yet: poll again from here
                excl += w[k] & LB_MASK;
                if (stt == LB_PREFIX) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            j -= k;  // tile 0 always publishes a prefix, so j stays >= 0
            if (k == 0 && (it & 63) == 63) {
                const unsigned long long tn = sort_gtimer();
                if (w0 == 0) {
                    w0 = tn;
                } else if (tn - w0 > wait_ns) {
                    gave_up = true;
                    break;
                }
            }
        }
    }
    // A wait that ran out: the block recounts every digit of its
    // predecessors straight from this pass's input (a permutation of the
    // keys, so the counts are exact), which keeps the pass correct and every
    // write inside the segment; the call still reports GEEK_ERR_TIMEOUT.
    if (__syncthreads_or(gave_up)) {
        if (t == 0) atomicExch(err, (int)GEEK_ERR_TIMEOUT);
        gbase[t] = 0;
        __syncthreads();
        const uint64_t *src = dsel ? hi_in : lo_in;
        for (int64_t p = t; p < t0; p += RS_THREADS) atomicAdd(&gbase[(uint32_t)((src[so + p] >> sh) & 0xFFu)], 1u);
        __syncthreads();
        excl = gbase[t];
        __syncthreads();
    }
    if (tile > 0 && tile != stall_tile) vlk[(int64_t)tile * 256 + t] = LB_PREFIX | ((excl + run) & LB_MASK);
    // output position of staged element q of digit d: goff[d] + q
    gbase[t] = dbase[(int64_t)seg * dstride + t] + excl - tstart[t];
    __syncthreads();
    const int cnt = (int)min((int64_t)RS_TILE, m - t0);
    for (int q = t; q < cnt; q += RS_THREADS) {
        const uint64_t kl = st_lo[q];
        const uint64_t kh = HI ? st_hi[q] : 0;
        const uint32_t d = (uint32_t)(((dsel ? kh : kl) >> sh) & 0xFFu);
        const int64_t dst = so + (uint32_t)(gbase[d] + (uint32_t)q);
        lo_out[dst] = kl;
        if (HI) hi_out[dst] = kh;
        if (VALS) v_out[dst] = st_v[q];
    }
}

// ---- run detection ---------------------------------------------------------
// a run starts where the key (lo, hi) or the optional tag changes
__device__ __forceinline__ bool run_start_at(const uint64_t *lo, const uint64_t *hi, const uint32_t *tag, int64_t p) {
    if (p == 0) return true;
    if (lo[p] != lo[p - 1]) return true;
    if (tag != nullptr && tag[p] != tag[p - 1]) return true;
    return hi != nullptr && hi[p] != hi[p - 1];
}

__global__ void __launch_bounds__(RS_THREADS) k_runs_count(const uint64_t *__restrict__ lo,
                                                           const uint64_t *__restrict__ hi,
                                                           const uint32_t *__restrict__ tag,
                                                           int64_t m, int tiles,
                                                           uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wsum[32];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const uint64_t *l = lo + (int64_t)seg * m;
    const uint64_t *h = hi ? hi + (int64_t)seg * m : nullptr;
    const uint32_t *g = tag ? tag + (int64_t)seg * m : nullptr;
    const int64_t p0 = (int64_t)tile * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
    uint32_t c = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t p = p0 + i;
        if (p < m && run_start_at(l, h, g, p)) c++;
    }
    uint32_t tot;
    block_excl_scan<RS_THREADS>(c, &tot, wsum);
    if (threadIdx.x == 0) tile_cnt[(int64_t)seg * tiles + tile] = tot;
}

__global__ void __launch_bounds__(RS_THREADS)
    k_runs_emit(const uint64_t *__restrict__ lo, const uint64_t *__restrict__ hi, const uint32_t *__restrict__ tag,
                int64_t m, int tiles, const uint32_t *__restrict__ tile_off, const int64_t *__restrict__ runs,
                int32_t *__restrict__ rank, int64_t *__restrict__ run_start) {
    __shared__ uint32_t wsum[32];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const uint64_t *l = lo + (int64_t)seg * m;
    const uint64_t *h = hi ? hi + (int64_t)seg * m : nullptr;
    const uint32_t *g = tag ? tag + (int64_t)seg * m : nullptr;
    int64_t *rs = run_start + (int64_t)seg * (m + 1);
    const int64_t p0 = (int64_t)tile * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
    uint32_t flags = 0, c = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t p = p0 + i;
        if (p < m && run_start_at(l, h, g, p)) {
            flags |= 1u << i;
            c++;
        }
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<RS_THREADS>(c, &tot, wsum) + tile_off[(int64_t)seg * tiles + tile];
    // rank of position p = (number of starts at positions <= p) - 1
    int64_t r = (int64_t)ex - 1;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t p = p0 + i;
        if (p >= m) break;
        if (flags >> i & 1u) {
            r++;
            rs[r] = p;
        }
        if (rank) rank[(int64_t)seg * m + p] = (int32_t)r;
    }
    if (tile == 0 && threadIdx.x == 0) rs[runs[seg]] = m;
}

// Bucket formation from sorted segments in one pass: position p of segment
// seg (key-sorted, ids[] the object ids in that order) belongs to run r;
// the object's bucket id in its table is r, and a run start records the
// run's global offset.  Writes obj_bucket[seg][ids[p]] = r and, at starts,
// boff[base[seg] + r] = seg * m + p; boff[NB] = S * m closes the list.
// The tile's keys and ids are first copied to shared memory with coalesced
// loads (a thread then walks RS_ITEMS consecutive positions there); the key
// before the tile comes along for the first run-start test.
__global__ void __launch_bounds__(RS_THREADS)
    k_runs_buckets(const uint64_t *__restrict__ lo, const uint64_t *__restrict__ hi, int64_t m, int tiles,
                   const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ ids,
                   const int64_t *__restrict__ base, int32_t *__restrict__ obj_bucket,
                   int64_t *__restrict__ boff, int64_t NB) {
    extern __shared__ uint64_t rb_sm[];  // lo [RS_TILE + 1], hi [RS_TILE + 1] (when hi), ids [RS_TILE]
    __shared__ uint32_t wsum[32];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const int64_t so = (int64_t)seg * m;
    const uint64_t *l = lo + so;
    const uint64_t *h = hi ? hi + so : nullptr;
    uint64_t *sl = rb_sm, *sh = rb_sm + (RS_TILE + 1);
    uint32_t *sid = reinterpret_cast<uint32_t *>(rb_sm + (h ? 2 : 1) * (RS_TILE + 1));
    const int64_t t0 = (int64_t)tile * RS_TILE;
    const int cnt = (int)min((int64_t)RS_TILE, m - t0);
    for (int e = threadIdx.x; e < cnt; e += RS_THREADS) {
        sl[e + 1] = l[t0 + e];
        if (h) sh[e + 1] = h[t0 + e];
        sid[e] = ids[so + t0 + e];
    }
    if (threadIdx.x == 0 && t0 > 0) {
        sl[0] = l[t0 - 1];
        if (h) sh[0] = h[t0 - 1];
    }
    __syncthreads();
    const int e0 = threadIdx.x * RS_ITEMS;
    uint32_t flags = 0, c = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        const int e = e0 + i;
        if (e < cnt && (t0 + e == 0 || sl[e + 1] != sl[e] || (h && sh[e + 1] != sh[e]))) {
            flags |= 1u << i;
            c++;
        }
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan<RS_THREADS>(c, &tot, wsum) + tile_off[(int64_t)seg * tiles + tile];
    int64_t r = (int64_t)ex - 1;
    const int64_t bb = base[seg];
    for (int i = 0; i < RS_ITEMS; i++) {
        const int e = e0 + i;
        if (e >= cnt) break;
        if (flags >> i & 1u) {
            r++;
            boff[bb + r] = so + t0 + e;
        }
        obj_bucket[so + sid[e]] = (int32_t)r;
    }
    if (seg == 0 && tile == 0 && threadIdx.x == 0) boff[NB] = (int64_t)gridDim.y * m;
}

// ---- generic int64 exclusive scan -----------------------------------------
__global__ void __launch_bounds__(RS_THREADS) k_i64_tile_sum(const int64_t *__restrict__ in,
                                                             int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t red[RS_THREADS];
    // the tile's sum in any order (integers): lane-contiguous, coalesced loads
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    int64_t s = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        const int64_t p = t0 + (int64_t)i * RS_THREADS + threadIdx.x;
        if (p < n) s += in[p];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = RS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// single block: exclusive scan of `n` int64 in place, total -> *total
__global__ void __launch_bounds__(1024) k_i64_scan_small(int64_t *__restrict__ a, int64_t n,
                                                         int64_t *__restrict__ total) {
    __shared__ int64_t buf[1024];
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t p = base + threadIdx.x;
        int64_t v = p < n ? a[p] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int64_t y = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (p < n) a[p] = carry + buf[threadIdx.x] - v;
        carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(RS_THREADS) k_i64_tile_apply(const int64_t *__restrict__ in,
                                                               int64_t *__restrict__ out, int64_t n,
                                                               const int64_t *__restrict__ sums) {
    __shared__ int64_t red[RS_THREADS];
    __shared__ int64_t tv[RS_TILE];  // the tile, loaded and stored coalesced
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    const int cnt = (int)min((int64_t)RS_TILE, n - t0);
    for (int e = threadIdx.x; e < RS_TILE; e += RS_THREADS) tv[e] = e < cnt ? in[t0 + e] : 0;
    __syncthreads();
    const int e0 = threadIdx.x * RS_ITEMS;
    int64_t v[RS_ITEMS];
    int64_t s = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        v[i] = tv[e0 + i];
        s += v[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 256 thread sums
    for (int o = 1; o < RS_THREADS; o <<= 1) {
        int64_t y = threadIdx.x >= o ? red[threadIdx.x - o] : 0;
        __syncthreads();
        red[threadIdx.x] += y;
        __syncthreads();
    }
    int64_t ex = red[threadIdx.x] - s + sums[blockIdx.x];
    for (int i = 0; i < RS_ITEMS; i++) {
        tv[e0 + i] = ex;
        ex += v[i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += RS_THREADS) out[t0 + e] = tv[e];
}

__global__ void k_iota_u32(uint32_t *v, int64_t n, int64_t period) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)(i % period);
}

}  // namespace

geek_status set_error(geek_ctx *ctx, geek_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

geek_status sort_err_word(geek_ctx *ctx) {
    if (ctx->sort_err) return GEEK_OK;
    GK_CUDA(ctx, cudaMalloc((void **)&ctx->sort_err, sizeof(int)));
    GK_CUDA(ctx, cudaMemset(ctx->sort_err, 0, sizeof(int)));
    return GEEK_OK;
}

geek_status sort_err_fetch(geek_ctx *ctx, int *h, cudaStream_t st) {
    *h = 0;
    if (!ctx->sort_err || ctx->capturing) return GEEK_OK;
    GK_CUDA(ctx, cudaMemcpyAsync(h, ctx->sort_err, sizeof *h, cudaMemcpyDeviceToHost, st));
    return GEEK_OK;
}

geek_status sort_err_eval(geek_ctx *ctx, const int *h, cudaStream_t st) {
    if (!*h) return GEEK_OK;
    GK_CUDA(ctx, cudaMemsetAsync(ctx->sort_err, 0, sizeof(int), st));
    return set_error(ctx, (geek_status)*h, "radix sort: a look-back wait timed out");
}

geek_status sort_err_check(geek_ctx *ctx, cudaStream_t st) {
    if (ctx->capturing) return GEEK_OK;
    int h = 0;
    GK_TRY(sort_err_fetch(ctx, &h, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    return sort_err_eval(ctx, &h, st);
}

void launch_iota_u32(uint32_t *v, int64_t n, int64_t period, cudaStream_t st) {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 1 << 16);
    GK_COUNT();
    k_iota_u32<<<blocks, 256, 0, st>>>(v, n, period);
}

geek_status radix_sort_segments(geek_ctx *ctx, Scratch &scr, int S, int64_t m, uint64_t **key_lo,
                                uint64_t **key_hi, uint32_t **vals, int nbits, cudaStream_t st) {
    if (S <= 0 || m <= 1 || nbits <= 0) return GEEK_OK;
    if (S > 65535) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "radix sort: %d segments", S);
    if (m > (int64_t)LB_MASK) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "radix sort: segment too long");
    if ((int64_t)S * ceil_div(m, RS_TILE) > 0xFFFFFFFFLL)
        return set_error(ctx, GEEK_ERR_UNSUPPORTED, "radix sort: too many tiles");
    const bool hi = nbits > 64;
    if (hi && !(key_hi && *key_hi)) return set_error(ctx, GEEK_ERR_INVALID, "radix sort: missing hi word");
    const bool hv = vals && *vals;
    const int tiles = (int)ceil_div(m, RS_TILE);
    const int64_t total = (int64_t)S * m;
    uint64_t *lo2 = nullptr, *hi2 = nullptr;
    uint32_t *v2 = nullptr;
    GK_TRY(scr.alloc(&lo2, total));
    if (hi) GK_TRY(scr.alloc(&hi2, total));
    if (hv) GK_TRY(scr.alloc(&v2, total));
    uint64_t *alo = *key_lo, *ahi = hi ? *key_hi : nullptr, *blo = lo2, *bhi = hi2;
    uint32_t *av = hv ? *vals : nullptr, *bv = v2;
    int passes = 0;
    const size_t stage = (size_t)RS_TILE * ((hi ? 16 : 8) + (hv ? 4 : 0));
    static bool attr_done = false;
    if (!attr_done) {
        const int mx = RS_TILE * 20;
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_onesweep<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_onesweep<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_onesweep<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_onesweep<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_hist_all, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 16 * 256 * 4));
        attr_done = true;
    }
    const int npass = (nbits + 7) / 8;
    // all digit offsets from one read of the keys
    uint32_t *dbase_all, *look, *ticket;
    GK_TRY(scr.alloc(&dbase_all, (size_t)S * npass * 256));
    GK_TRY(scr.alloc(&look, (size_t)S * tiles * 256 + 32));
    ticket = look + (size_t)S * tiles * 256;
    GK_TRY(sort_err_word(ctx));
    GK_CUDA(ctx, cudaMemsetAsync(dbase_all, 0, sizeof(uint32_t) * S * npass * 256, st));
    {
        const int hb = (int)std::min<int64_t>(HIST_BLOCKS_PER_SEG, ceil_div(m, 256 * 16));
        GK_COUNT();
        k_rs_hist_all<<<dim3(std::max(hb, 1), S), 256, (size_t)4 * npass * 256 * 4, st>>>(alo, hi ? ahi : nullptr, m, npass,
                                                                                        dbase_all);
        GK_LAUNCH(ctx);
        GK_COUNT();
        k_rs_base_all<<<S * npass, 256, 0, st>>>(dbase_all);
        GK_LAUNCH(ctx);
    }
    const int64_t nblocks = (int64_t)S * tiles;
    for (int q = 0; q < npass; q++, passes++) {
        const int sh = q * 8, dsel = sh >= 64, sv = sh & 63;
        GK_CUDA(ctx, cudaMemsetAsync(look, 0, sizeof(uint32_t) * ((size_t)S * tiles * 256 + 32), st));
        EvTimer tk(ctx, "kernel.rs_scatter", st);
        tk.work = 2.0 * (double)total * ((hi ? 16 : 8) + (hv ? 4 : 0));
        GK_COUNT();
#define RS_OS(H, V)                                                                                              \
    k_rs_onesweep<H, V><<<(unsigned)nblocks, RS_THREADS, stage, st>>>(alo, ahi, av, blo, bhi, bv, m, tiles, dsel, sv, \
                                                                      dbase_all + (size_t)q * 256, npass * 256, look, \
                                                                      ticket, ctx->sort_err, ctx->lb_wait_ns, ctx->stall_tile)
        if (hi && hv) RS_OS(true, true);
        else if (hi) RS_OS(true, false);
        else if (hv) RS_OS(false, true);
        else RS_OS(false, false);
#undef RS_OS
        GK_LAUNCH(ctx);
        std::swap(alo, blo);
        std::swap(ahi, bhi);
        std::swap(av, bv);
    }
    if (passes & 1) {  // result lives in the scratch buffers: copy back
        GK_CUDA(ctx, cudaMemcpyAsync(*key_lo, alo, total * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        if (hi) GK_CUDA(ctx, cudaMemcpyAsync(*key_hi, ahi, total * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        if (hv) GK_CUDA(ctx, cudaMemcpyAsync(*vals, av, total * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    return GEEK_OK;
}

geek_status segment_runs(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                         const uint64_t *key_hi, int32_t *rank, int64_t *run_start, int64_t *runs,
                         cudaStream_t st) {
    return segment_runs_tagged(ctx, scr, S, m, key_lo, key_hi, nullptr, rank, run_start, runs, st);
}

geek_status segment_runs_tagged(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                                const uint64_t *key_hi, const uint32_t *tag, int32_t *rank, int64_t *run_start,
                                int64_t *runs, cudaStream_t st) {
    if (S <= 0) return GEEK_OK;
    if (m == 0) {
        GK_CUDA(ctx, cudaMemsetAsync(runs, 0, sizeof(int64_t) * S, st));
        GK_CUDA(ctx, cudaMemsetAsync(run_start, 0, sizeof(int64_t) * S, st));
        return GEEK_OK;
    }
    const int tiles = (int)ceil_div(m, RS_TILE);
    uint32_t *tile_cnt;
    GK_TRY(scr.alloc(&tile_cnt, (size_t)S * tiles));
    const dim3 grid(tiles, S);
    GK_COUNT();
    k_runs_count<<<grid, RS_THREADS, 0, st>>>(key_lo, key_hi, tag, m, tiles, tile_cnt);
    GK_COUNT();
    k_seg_scan_u32<<<S, 1024, 0, st>>>(tile_cnt, tiles, runs);
    GK_COUNT();
    k_runs_emit<<<grid, RS_THREADS, 0, st>>>(key_lo, key_hi, tag, m, tiles, tile_cnt, runs, rank, run_start);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status segment_buckets(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                            const uint64_t *key_hi, const uint32_t *ids, int32_t *obj_bucket, int64_t **boff_out,
                            std::vector<int64_t> &nb, int64_t *NB_out, cudaStream_t st) {
    nb.assign(S, 0);
    int64_t *runs;
    GK_TRY(scr.alloc(&runs, std::max(S, 1)));
    const int tiles = (int)std::max<int64_t>(1, ceil_div(m, RS_TILE));
    uint32_t *tile_cnt = nullptr;
    if (S > 0 && m > 0) {
        GK_TRY(scr.alloc(&tile_cnt, (size_t)S * tiles));
        GK_COUNT();
        k_runs_count<<<dim3(tiles, S), RS_THREADS, 0, st>>>(key_lo, key_hi, nullptr, m, tiles, tile_cnt);
        GK_COUNT();
        k_seg_scan_u32<<<S, 1024, 0, st>>>(tile_cnt, tiles, runs);
        GK_LAUNCH(ctx);
        GK_CUDA(ctx, cudaMemcpyAsync(nb.data(), runs, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, st));
    }
    int sort_err = 0;
    GK_TRY(sort_err_fetch(ctx, &sort_err, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    GK_TRY(sort_err_eval(ctx, &sort_err, st));
    std::vector<int64_t> base(std::max(S, 1), 0);
    int64_t NB = 0;
    for (int l = 0; l < S; l++) {
        base[l] = NB;
        NB += nb[l];
    }
    int64_t *boff;
    cudaError_t e = cudaMallocAsync((void **)&boff, sizeof(int64_t) * (NB + 1), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, GEEK_ERR_NOMEM, "bucket offsets: %s", cudaGetErrorString(e));
    }
    if (S == 0 || m == 0) {
        const int64_t sentinel = (int64_t)S * m;  // = 0
        GK_CUDA(ctx, cudaMemcpyAsync(boff + NB, &sentinel, sizeof sentinel, cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
    } else {
        int64_t *d_base;
        GK_TRY(scr.alloc(&d_base, S));
        GK_CUDA(ctx, cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, st));
        GK_COUNT();
        const size_t rb_smem = (size_t)(key_hi ? 2 : 1) * (RS_TILE + 1) * sizeof(uint64_t) + RS_TILE * sizeof(uint32_t);
        static bool rb_attr = false;
        if (!rb_attr) {
            GK_CUDA(ctx, cudaFuncSetAttribute(k_runs_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(2 * (RS_TILE + 1) * sizeof(uint64_t) + RS_TILE * sizeof(uint32_t))));
            rb_attr = true;
        }
        k_runs_buckets<<<dim3(tiles, S), RS_THREADS, rb_smem, st>>>(key_lo, key_hi, m, tiles, tile_cnt, ids, d_base,
                                                                   obj_bucket, boff, NB);
        GK_LAUNCH(ctx);
    }
    *boff_out = boff;
    *NB_out = NB;
    return GEEK_OK;
}

geek_status exclusive_scan_i64(geek_ctx *ctx, Scratch &scr, const int64_t *in, int64_t *out,
                               int64_t n, int64_t *total_dev, cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) GK_CUDA(ctx, cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st));
        return GEEK_OK;
    }
    const int64_t tiles = ceil_div(n, RS_TILE);
    int64_t *sums;
    GK_TRY(scr.alloc(&sums, tiles));
    GK_COUNT();
    k_i64_tile_sum<<<(unsigned)tiles, RS_THREADS, 0, st>>>(in, n, sums);
    GK_COUNT();
    k_i64_scan_small<<<1, 1024, 0, st>>>(sums, tiles, total_dev);
    GK_COUNT();
    k_i64_tile_apply<<<(unsigned)tiles, RS_THREADS, 0, st>>>(in, out, n, sums);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}
