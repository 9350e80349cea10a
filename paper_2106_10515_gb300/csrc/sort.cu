// Device radix sort, run detection and prefix sums: the grouping machinery
// behind bucket formation (T[G(x)].push(j) in Algs. 2-3), SILK bins (Alg. 4)
// and majority voting.  Sorting is a stable LSD radix sort with 8-bit digits
// over S equal-length segments at once (one segment per hash table), so the
// L tables of a transform share every launch.
#include <cstdarg>

#include "common.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 elements per tile
constexpr int NWARP = RS_THREADS / 32;

// ---- histogram of one digit per (segment, tile) ---------------------------
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ word, int sh,
                                                        int64_t m, int tiles,
                                                        uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[256];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const uint32_t lane = t & 31;
    h[t] = 0;
    __syncthreads();
    const uint64_t *w = word + (int64_t)seg * m;
    const int64_t base = (int64_t)tile * RS_TILE;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t p = base + (int64_t)i * RS_THREADS + t;
        uint32_t dg = p < m ? (uint32_t)(w[p] >> sh) & 0xFFu : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256 && (peers & ((1u << lane) - 1)) == 0) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[((int64_t)seg * 256 + t) * tiles + tile] = h[t];
}

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

// Digit offsets of one radix pass.  counts is [S][256][tiles]; one block per
// (segment, digit) turns its tile counts into an exclusive scan and records
// the digit total; k_digit_base then scans the 256 totals of each segment.
__global__ void __launch_bounds__(1024) k_digit_tile_scan(uint32_t *__restrict__ counts, int tiles,
                                                          uint32_t *__restrict__ dtot) {
    __shared__ uint32_t wsum[32];
    const int seg = blockIdx.y, dg = blockIdx.x;
    uint32_t *a = counts + ((int64_t)seg * 256 + dg) * tiles;
    uint32_t carry = 0;
    for (int base = 0; base < tiles; base += 1024) {
        const int p = base + threadIdx.x;
        const uint32_t v = p < tiles ? a[p] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<1024>(v, &tot, wsum) + carry;
        if (p < tiles) a[p] = ex;
        carry += tot;
    }
    if (threadIdx.x == 0) dtot[seg * 256 + dg] = carry;
}

__global__ void __launch_bounds__(256) k_digit_base(uint32_t *__restrict__ dtot) {
    __shared__ uint32_t wsum[32];
    uint32_t *a = dtot + blockIdx.x * 256;
    const uint32_t v = a[threadIdx.x];
    uint32_t tot;
    const uint32_t ex = block_excl_scan<256>(v, &tot, wsum);
    a[threadIdx.x] = ex;
}

// ---- stable scatter of one digit ------------------------------------------
// A tile of 4096 elements is split into 8 warp slices of 512; warp w reads
// its slice striped (item i of lane l is element w*512 + i*32 + l), so the
// order (warp, item, lane) is the input order.  Each warp ranks its elements
// per digit with match-any (a running per-warp digit count in shared memory),
// the block turns the per-warp counts into tile offsets, the tile is staged
// in shared memory in (digit, input order), and written out contiguously per
// digit: coalesced stores, stable order, three block barriers per tile.
// (3 blocks per SM: the scatter is latency bound, and occupancy is worth
// the few registers spilled)
template <bool HI, bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 3)
    k_rs_scatter(const uint64_t *__restrict__ lo_in, const uint64_t *__restrict__ hi_in,
                 const uint32_t *__restrict__ v_in, uint64_t *__restrict__ lo_out,
                 uint64_t *__restrict__ hi_out, uint32_t *__restrict__ v_out, int64_t m, int tiles,
                 int dsel, int sh, const uint32_t *__restrict__ offs, const uint32_t *__restrict__ dbase) {
    __shared__ uint32_t whist[NWARP][256];
    __shared__ uint32_t tstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[32];
    extern __shared__ uint64_t stage[];
    uint64_t *st_lo = stage;
    uint64_t *st_hi = stage + RS_TILE;
    uint32_t *st_v = (uint32_t *)(stage + (HI ? 2 : 1) * RS_TILE);
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t so = (int64_t)seg * m;
    const int64_t t0 = (int64_t)tile * RS_TILE;
    const uint32_t lt = (1u << lane) - 1;
#pragma unroll
    for (int w = 0; w < NWARP; w++) whist[w][t] = 0;
    gbase[t] = offs[((int64_t)seg * 256 + t) * tiles + tile] + dbase[seg * 256 + t];
    __syncthreads();
    constexpr int IT = RS_TILE / RS_THREADS;  // 16 items per lane
    uint64_t klo[IT], khi[IT];
    uint32_t vv[IT], dr[IT];  // dr = digit | rank-in-warp << 9
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int64_t p = t0 + warp * (IT * 32) + i * 32 + lane;
        const bool valid = p < m;
        klo[i] = valid ? lo_in[so + p] : 0;
        khi[i] = (HI && valid) ? hi_in[so + p] : 0;
        vv[i] = (VALS && valid) ? v_in[so + p] : 0;
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
    __syncthreads();
    const int cnt = (int)min((int64_t)RS_TILE, m - t0);
    for (int q = t; q < cnt; q += RS_THREADS) {
        const uint64_t kl = st_lo[q];
        const uint64_t kh = HI ? st_hi[q] : 0;
        const uint32_t d = (uint32_t)(((dsel ? kh : kl) >> sh) & 0xFFu);
        const int64_t dst = so + gbase[d] + (q - tstart[d]);
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

// ---- generic int64 exclusive scan -----------------------------------------
__global__ void __launch_bounds__(RS_THREADS) k_i64_tile_sum(const int64_t *__restrict__ in,
                                                             int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t red[RS_THREADS];
    const int64_t p0 = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
    int64_t s = 0;
    for (int i = 0; i < RS_ITEMS; i++)
        if (p0 + i < n) s += in[p0 + i];
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
    const int64_t p0 = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
    int64_t v[RS_ITEMS];
    int64_t s = 0;
    for (int i = 0; i < RS_ITEMS; i++) {
        v[i] = p0 + i < n ? in[p0 + i] : 0;
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
        if (p0 + i < n) out[p0 + i] = ex;
        ex += v[i];
    }
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
    if (m > 0xFFFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "radix sort: segment too long");
    const bool hi = nbits > 64;
    if (hi && !(key_hi && *key_hi)) return set_error(ctx, GEEK_ERR_INVALID, "radix sort: missing hi word");
    const bool hv = vals && *vals;
    const int tiles = (int)ceil_div(m, RS_TILE);
    const int64_t total = (int64_t)S * m;
    uint32_t *counts, *dtot;
    GK_TRY(scr.alloc(&counts, (size_t)S * 256 * tiles));
    GK_TRY(scr.alloc(&dtot, (size_t)S * 256));
    uint64_t *lo2 = nullptr, *hi2 = nullptr;
    uint32_t *v2 = nullptr;
    GK_TRY(scr.alloc(&lo2, total));
    if (hi) GK_TRY(scr.alloc(&hi2, total));
    if (hv) GK_TRY(scr.alloc(&v2, total));
    uint64_t *alo = *key_lo, *ahi = hi ? *key_hi : nullptr, *blo = lo2, *bhi = hi2;
    uint32_t *av = hv ? *vals : nullptr, *bv = v2;
    int passes = 0;
    const dim3 grid(tiles, S);
    const size_t stage = (size_t)RS_TILE * ((hi ? 16 : 8) + (hv ? 4 : 0));
    static bool attr_done = false;
    if (!attr_done) {
        const int mx = RS_TILE * 20;
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_scatter<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_scatter<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_scatter<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        GK_CUDA(ctx, cudaFuncSetAttribute(k_rs_scatter<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        attr_done = true;
    }
    for (int sh = 0; sh < nbits; sh += 8, passes++) {
        const int dsel = sh >= 64, s = sh & 63;
        GK_COUNT();
        k_rs_hist<<<grid, RS_THREADS, 0, st>>>(dsel ? ahi : alo, s, m, tiles, counts);
        GK_COUNT();
        k_digit_tile_scan<<<dim3(256, S), 1024, 0, st>>>(counts, tiles, dtot);
        GK_COUNT();
        k_digit_base<<<S, 256, 0, st>>>(dtot);
        EvTimer tk(ctx, "kernel.rs_scatter", st);
        tk.work = 2.0 * (double)total * ((hi ? 16 : 8) + (hv ? 4 : 0));
        GK_COUNT();
        if (hi && hv)
            k_rs_scatter<true, true><<<grid, RS_THREADS, stage, st>>>(alo, ahi, av, blo, bhi, bv, m, tiles, dsel, s, counts, dtot);
        else if (hi)
            k_rs_scatter<true, false><<<grid, RS_THREADS, stage, st>>>(alo, ahi, av, blo, bhi, bv, m, tiles, dsel, s, counts, dtot);
        else if (hv)
            k_rs_scatter<false, true><<<grid, RS_THREADS, stage, st>>>(alo, ahi, av, blo, bhi, bv, m, tiles, dsel, s, counts, dtot);
        else
            k_rs_scatter<false, false><<<grid, RS_THREADS, stage, st>>>(alo, ahi, av, blo, bhi, bv, m, tiles, dsel, s, counts, dtot);
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
