// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "geek.h"

#define GEEK_VERSION_STRING "geek-gb300 0.1 (sm_103a)"

struct geek_ctx {
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    // CUDA-event timing of phases and kernels (off by default)
    bool timing = false;
    bool capturing = false;  // a stream capture is open: no event brackets
    struct Timed {
        double ms = 0.0;
        long long count = 0;
        double work = 0.0;  // algorithmic bytes or flops of the bracketed work
    };
    mutable std::map<std::string, Timed> times;
    // brackets whose end event has been recorded but not yet read: resolved
    // (waited for and added to times) when the timings are read or reset, so
    // a bracket adds no host synchronisation to the work it measures
    struct Pending {
        const char *name;
        cudaEvent_t a, b;
        double work;
    };
    mutable std::vector<Pending> pending;
    void resolve_timers() const {
        for (const Pending &q : pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
                auto &e = times[q.name];
                e.ms += ms;
                e.count += 1;
                e.work += q.work;
            }
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        pending.clear();
    }
    // (centre-tile width | split-BF16 << 16) chosen by the batch autotuner per
    // (precision setting, padded d, seed-count class)
    std::map<int, int> tile_cache;
    // device word a bounded wait of the radix sort sets on timeout (lazy)
    int *sort_err = nullptr;
    // limit of one look-back wait of the radix passes (GEEK_OPT_WAIT_LIMIT_NS)
    unsigned long long lb_wait_ns = 2000000000ull;
    // failure injection (tests): a radix tile that never publishes its count
    // (GEEK_OPT_TEST_STALL_TILE, -1 off) and a countdown after which device
    // allocations fail (GEEK_OPT_TEST_FAIL_ALLOC, -1 off)
    int stall_tile = -1;
    long long fail_alloc_after = -1;
    ~geek_ctx() {
        for (const Pending &q : pending) {
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        if (sort_err) cudaFree(sort_err);
    }
};

// Brackets work on a stream with CUDA events when ctx->timing is on; the
// event pair is queued on the context when the bracket ends and its elapsed
// time added to ctx->times[name] when the timings are read (no wait here).
struct EvTimer {
    geek_ctx *ctx;
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    double work = 0.0;
    EvTimer(geek_ctx *c, const char *nm, cudaStream_t s) : ctx(c), name(nm), st(s) {
        if (ctx && ctx->timing && !ctx->capturing && cudaEventCreate(&a) == cudaSuccess &&
            cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, st);
    }
    void stop() {
        if (!b) return;
        cudaEventRecord(b, st);
        ctx->pending.push_back(geek_ctx::Pending{name, a, b, work});
        a = b = nullptr;
    }
    ~EvTimer() { stop(); }
};

// Failure injection of GEEK_OPT_TEST_FAIL_ALLOC: true when this allocation
// is to fail (the countdown reached zero); the countdown then stays off.
static inline bool alloc_injected_failure(geek_ctx *ctx) {
    if (!ctx || ctx->fail_alloc_after < 0) return false;
    if (ctx->fail_alloc_after == 0) {
        ctx->fail_alloc_after = -1;
        return true;
    }
    ctx->fail_alloc_after--;
    return false;
}

// Per-call error plumbing: every failure sets ctx->last_error and returns.
geek_status set_error(geek_ctx *ctx, geek_status st, const char *fmt, ...);

#define GK_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_error((ctx), e_ == cudaErrorMemoryAllocation ? GEEK_ERR_NOMEM         \
                                                                    : GEEK_ERR_CUDA,         \
                             "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),         \
                             __FILE__, __LINE__);                                            \
    } while (0)

#define GK_TRY(expr)                                                                         \
    do {                                                                                     \
        geek_status s_ = (expr);                                                             \
        if (s_ != GEEK_OK) return s_;                                                        \
    } while (0)

#define GK_LAUNCH(ctx) GK_CUDA(ctx, cudaGetLastError())

// Number of kernels this library has launched (process-wide), read through
// geek_launch_count() by callers that account for device work.
extern unsigned long long g_geek_launches;
#define GK_COUNT() (__atomic_fetch_add(&g_geek_launches, 1ull, __ATOMIC_RELAXED))

// Stream-ordered scratch owned by one API call; freed (stream-ordered) when
// the call returns.
struct Scratch {
    geek_ctx *ctx;
    cudaStream_t st;
    std::vector<void *> ptrs;
    Scratch(geek_ctx *c, cudaStream_t s) : ctx(c), st(s) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
    template <class T>
    geek_status alloc(T **out, size_t count) {
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (alloc_injected_failure(ctx))
            return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed (injected)", bytes);
        cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed: %s", bytes,
                             cudaGetErrorString(e));
        }
        ptrs.push_back(p);
        *out = (T *)p;
        return GEEK_OK;
    }
    // hands the allocation to the caller (it will not be freed here)
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) q = nullptr;
    }
};

// Device buffer owned by a result handle.
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
};

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static inline int bit_length_u64(uint64_t v) {
    int b = 0;
    while (v) {
        b++;
        v >>= 1;
    }
    return b;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Multiply-add-shift hash standing in for MinHash's random permutation
// (Eq. 2): floor(((A*x + B) mod 2^64) / 2^32), computed from 32-bit halves:
// the low 64 bits of A*x equal lo32(A)*x + (hi32(A)*x mod 2^32) * 2^32.
__device__ __forceinline__ uint32_t mh_hash32(uint64_t A, uint64_t B, uint32_t x) {
    uint64_t t = (uint64_t)(uint32_t)A * (uint64_t)x + B;
    uint32_t hi = (uint32_t)(t >> 32) + (uint32_t)(A >> 32) * x;
    return hi;
}

// Largest i < count with off[i] <= v: the instance (or block range) holding
// global index v, for ascending offsets off[0..count] (empty ranges are
// skipped because a later equal offset wins).
static __device__ __forceinline__ int find_inst(const int64_t *__restrict__ off, int count, int64_t v) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Internal building blocks (implemented in the .cu files)
// ---------------------------------------------------------------------------

// Allocates ctx->sort_err (zeroed) on first use.
geek_status sort_err_word(geek_ctx *ctx);
// Synchronises `st`, then reads and clears ctx->sort_err (no-op while
// capturing):
// TIMEOUT when a radix pass gave up waiting on a predecessor tile.
geek_status sort_err_check(geek_ctx *ctx, cudaStream_t st);
// The same in two halves around a synchronisation the caller makes anyway:
// fetch enqueues the copy into *h, eval (after the sync) clears and reports.
geek_status sort_err_fetch(geek_ctx *ctx, int *h, cudaStream_t st);
geek_status sort_err_eval(geek_ctx *ctx, const int *h, cudaStream_t st);

// Stable LSD radix sort of S segments of m elements each (m < 2^30).  Keys are up to
// 128 bits: key_lo holds bits 0..63, key_hi (may be null when nbits <= 64)
// bits 64..127.  vals (may be null) moves with the keys.  Only bits
// [0, nbits) are examined.  On return the sorted data is in the buffers
// pointed to by *key_lo / *key_hi / *vals (which may have been swapped with
// internal buffers allocated from `scr`).
geek_status radix_sort_segments(geek_ctx *ctx, Scratch &scr, int S, int64_t m, uint64_t **key_lo,
                                uint64_t **key_hi, uint32_t **vals, int nbits, cudaStream_t st);

// Buckets of S key-sorted segments of m elements (ids: object id at each
// sorted position): obj_bucket[seg][id] = rank of the id's key among the
// segment's distinct keys; *boff_out (stream-ordered allocation, NB + 1
// entries) holds the global start seg * m + p of every run, tables in order,
// then S * m; nb[seg] = runs of segment seg, *NB_out their sum.  Synchronises
// `st` once (the run counts size the offsets) and reports a radix-sort
// timeout recorded before it.
geek_status segment_buckets(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                            const uint64_t *key_hi, const uint32_t *ids, int32_t *obj_bucket, int64_t **boff_out,
                            std::vector<int64_t> &nb, int64_t *NB_out, cudaStream_t st);

// Run detection over S segments of m sorted keys: starts flagged where the
// key differs from its predecessor in the segment.  Produces
//   rank[p]         (may be null)  run index of position p within its segment
//   run_start[s*(m+1) + r]         position of run r in segment s (r < runs[s]),
//                                  and run_start[s*(m+1) + runs[s]] = m
//   runs[s]                        runs in segment s (device)
geek_status segment_runs(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                         const uint64_t *key_hi, int32_t *rank, int64_t *run_start, int64_t *runs,
                         cudaStream_t st);
// As segment_runs, with an optional tag per position (S x m, may be null):
// a run also starts where the tag changes.
geek_status segment_runs_tagged(geek_ctx *ctx, Scratch &scr, int S, int64_t m, const uint64_t *key_lo,
                                const uint64_t *key_hi, const uint32_t *tag, int32_t *rank, int64_t *run_start,
                                int64_t *runs, cudaStream_t st);

// Exclusive prefix sum of n int64 values (in place allowed); total -> *total_dev.
geek_status exclusive_scan_i64(geek_ctx *ctx, Scratch &scr, const int64_t *in, int64_t *out,
                               int64_t n, int64_t *total_dev, cudaStream_t st);

// iota fill
void launch_iota_u32(uint32_t *v, int64_t n, int64_t period, cudaStream_t st);
