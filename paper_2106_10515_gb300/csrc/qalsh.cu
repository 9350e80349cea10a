// Alg. 1 (Sect. 3.1, homogeneous dense data): m QALSH projections
// s = a_f . x, each table sorted by (s, object id) and cut into t parts of
// sizes floor((j + 1) n / t) - floor(j n / t).
//
// The projections run in FP32 (the register-tiled projection kernel, raw
// epilogue); the FP32 order is exact everywhere except near the cuts.  With
// E = d * 6e-8 |a_f| max_i |x_i| >= |v_i - s_i| for every object (v the FP32
// value, s the pinned FP64 dot product), the exact value tau at cut position
// p lies within E of the FP32 value there (order statistics move by at most
// the largest perturbation).  So every object whose FP32 value is more than
// 2E below (above) v_(p) is exactly before (after) the cut, and only the
// objects in the window [v_(p) - 2E, v_(p) + 2E] of the FP32 order can
// change sides: their FP64 values are computed and each window (windows
// that overlap are merged) is re-sorted by (s, id).  Outside the windows the
// FP32 position already gives the exact part.
#include <algorithm>

#include "internal.cuh"

namespace {

// order-preserving unsigned keys of IEEE values
__device__ __forceinline__ uint32_t f32_key(uint32_t u) { return (u & 0x80000000u) ? ~u : (u | 0x80000000u); }
__device__ __forceinline__ float key_f32(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ uint64_t f64_key(double v) {
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | (1ull << 63));
}

// keys[f][i] = key of the FP32 value vals[i][f]; ids[f][i] = i
__global__ void k_qalsh_keys(int64_t n, int m, const float *__restrict__ vals, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *vr = vals + i * m;
        for (int f = 0; f < m; f++) {
            keys[(int64_t)f * n + i] = f32_key(__float_as_uint(vr[f]));
            ids[(int64_t)f * n + i] = (uint32_t)i;
        }
    }
}

// first index in the ascending keys k[0..n) with k >= v (upper: k > v)
__device__ __forceinline__ int64_t lower_key(const uint64_t *k, int64_t n, uint64_t v, bool upper) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (upper ? k[mid] <= v : k[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// window of cut j (1 .. t-1) of table f: FP32-sorted positions whose value is
// within 2.01 E of the value at the cut position floor(j n / t)
__global__ void k_qalsh_windows(int64_t n, int m, int t, const uint64_t *__restrict__ keys,
                                const float *__restrict__ anorm, const unsigned *__restrict__ xmax_bits, double gam,
                                int64_t *__restrict__ q0, int64_t *__restrict__ q1) {
    const int64_t tot = (int64_t)m * (t - 1);
    const double xm = (double)__uint_as_float(*xmax_bits);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / (t - 1));
        const int64_t j = e % (t - 1) + 1;
        const int64_t p = j * n / t;
        const uint64_t *kf = keys + (int64_t)f * n;
        const double v = (double)key_f32((uint32_t)kf[p]);
        const double E = gam * (double)anorm[f] * xm;
        float lo = __double2float_rd(v - 2.01 * E), hi = __double2float_ru(v + 2.01 * E);
        if (lo == 0.f) lo = -0.f;  // -0 and +0 are equal values: take both
        if (hi == 0.f) hi = 0.f;
        q0[e] = lower_key(kf, n, f32_key(__float_as_uint(lo)), false);
        q1[e] = lower_key(kf, n, f32_key(__float_as_uint(hi)), true);
    }
}

// one warp per merged window w (table wf[w], positions [wq0, wq1), list
// entries from woff[w]): the pinned FP64 dot product of every object in it,
// keyed (window, FP64 value, id) for one sort of all windows
__global__ void k_qalsh_gather(int64_t nwin, const int *__restrict__ wf, const int64_t *__restrict__ wq0,
                               const int64_t *__restrict__ wq1, const int64_t *__restrict__ woff,
                               const uint32_t *__restrict__ ids, int64_t n, const float *__restrict__ x, int64_t ldx,
                               int d, const float *__restrict__ a, uint64_t *__restrict__ klo,
                               uint64_t *__restrict__ khi) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nwin; w += nw) {
        const int f = wf[w];
        const int64_t q0 = wq0[w], len = wq1[w] - q0, off = woff[w];
        const float *af = a + (int64_t)f * d;
        for (int64_t r = lane; r < len; r += 32) {
            const uint32_t id = ids[(int64_t)f * n + q0 + r];
            const float *xr = x + (int64_t)id * ldx;
            double s = 0.0;
            for (int j = 0; j < d; j++) s = __dadd_rn(s, __dmul_rn((double)af[j], (double)xr[j]));
            const uint64_t k = f64_key(__dadd_rn(s, 0.0));  // -0 -> +0: equal values tie by id
            khi[off + r] = ((uint64_t)w << 32) | (k >> 32);
            klo[off + r] = (k << 32) | id;
        }
    }
}

// sorted list entry e back into its window: position wq0 + (e - woff)
__global__ void k_qalsh_put(int64_t W, const uint64_t *__restrict__ klo, const uint64_t *__restrict__ khi,
                            const int *__restrict__ wf, const int64_t *__restrict__ wq0,
                            const int64_t *__restrict__ woff, uint32_t *__restrict__ ids, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < W; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = (int64_t)(khi[e] >> 32);
        ids[(int64_t)wf[w] * n + wq0[w] + (e - woff[w])] = (uint32_t)klo[e];
    }
}

// part of sorted position p: the largest j with floor(j n / t) <= p
__global__ void k_qalsh_parts(int64_t n, int m, int t, const uint32_t *__restrict__ ids,
                              int32_t *__restrict__ obj_bucket) {
    const int f = blockIdx.y;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = ((p + 1) * t + n - 1) / n - 1;
        obj_bucket[(int64_t)f * n + ids[(int64_t)f * n + p]] = (int32_t)j;
    }
}

// members: objects in id order keyed by their part, stably sorted
__global__ void k_qalsh_member_keys(int64_t tot, int64_t n, const int32_t *__restrict__ obj_bucket,
                                    uint64_t *__restrict__ key, uint32_t *__restrict__ ids) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = (uint64_t)(uint32_t)obj_bucket[e];
        ids[e] = (uint32_t)(e % n);
    }
}

__global__ void k_qalsh_boff(int64_t n, int m, int t, int64_t *__restrict__ boff) {
    const int64_t tot = (int64_t)m * t;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= tot; e += (int64_t)gridDim.x * blockDim.x)
        boff[e] = e == tot ? (int64_t)m * n : (e / t) * n + (e % t) * n / t;
}

}  // namespace

geek_status hash_qalsh(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d, const float *a,
                       int m, int t, geek_buckets *b, cudaStream_t st) {
    if (m < 1 || m > 512) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "QALSH: 1 <= m <= 512 tables");
    if (n > 0 && (t < 1 || t > n)) return set_error(ctx, GEEK_ERR_INVALID, "QALSH: need 1 <= t <= n");
    if (n > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "QALSH: more than 2^31 objects");
    float *anorm;
    unsigned *xmax;
    GK_TRY(scr.alloc(&anorm, m));
    GK_TRY(scr.alloc(&xmax, 1));
    GK_TRY(project_raw(ctx, scr, x, ldx, n, d, a, m, (float *)b->codes, anorm, xmax, st));
    b->nb.assign(m, n > 0 ? t : 0);
    b->NB = n > 0 ? (int64_t)m * t : 0;
    b->key_bits_max = 32;
    GK_CUDA(ctx, cudaMallocAsync((void **)&b->boff, sizeof(int64_t) * (b->NB + 1), st));
    if (n == 0) {
        GK_CUDA(ctx, cudaMemsetAsync(b->boff, 0, sizeof(int64_t), st));
        return GEEK_OK;
    }
    const int64_t tot = n * m;
    uint64_t *keys;
    GK_TRY(scr.alloc(&keys, tot));
    uint32_t *ids = b->members;  // the FP32 order first, the members at the end
    GK_COUNT();
    k_qalsh_keys<<<grid_for(n, 256, ctx->num_sms), 256, 0, st>>>(n, m, (const float *)b->codes, keys, ids);
    GK_LAUNCH(ctx);
    {
        EvTimer tk(ctx, "hash.sort", st);
        GK_TRY(radix_sort_segments(ctx, scr, m, n, &keys, nullptr, &ids, 32, st));
    }
    if (t > 1) {
        const int64_t nc = (int64_t)m * (t - 1);
        int64_t *q0, *q1;
        GK_TRY(scr.alloc(&q0, nc));
        GK_TRY(scr.alloc(&q1, nc));
        const double gam = (double)d * 6.0e-8;  // as for E2LSH: >= gamma_d + d 2^-53 and the norms' error
        GK_COUNT();
        k_qalsh_windows<<<grid_for(nc, 256, ctx->num_sms), 256, 0, st>>>(n, m, t, keys, anorm, xmax, gam, q0, q1);
        GK_LAUNCH(ctx);
        std::vector<int64_t> h0(nc), h1(nc);
        GK_CUDA(ctx, cudaMemcpyAsync(h0.data(), q0, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaMemcpyAsync(h1.data(), q1, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, st));
        GK_TRY(sort_err_check(ctx, st));  // synchronises st
        // merge the overlapping windows of each table (cuts in order, so
        // window starts never decrease)
        std::vector<int> wf;
        std::vector<int64_t> w0, w1, wo;
        int64_t W = 0;
        for (int f = 0; f < m; f++) {
            int64_t c0 = -1, c1 = -1;
            for (int64_t j = 0; j < t - 1; j++) {
                const int64_t a0 = h0[(size_t)f * (t - 1) + j], a1 = h1[(size_t)f * (t - 1) + j];
                if (c0 >= 0 && a0 < c1) {
                    c1 = std::max(c1, a1);
                    continue;
                }
                if (c0 >= 0 && c1 > c0) {
                    wf.push_back(f);
                    w0.push_back(c0);
                    w1.push_back(c1);
                    wo.push_back(W);
                    W += c1 - c0;
                }
                c0 = a0;
                c1 = a1;
            }
            if (c0 >= 0 && c1 > c0) {
                wf.push_back(f);
                w0.push_back(c0);
                w1.push_back(c1);
                wo.push_back(W);
                W += c1 - c0;
            }
        }
        const int64_t nwin = (int64_t)wf.size();
        if (nwin >= 0xFFFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "QALSH: too many cut windows");
        if (W > 0) {
            int *d_wf;
            int64_t *d_w0, *d_w1, *d_wo;
            GK_TRY(scr.alloc(&d_wf, nwin));
            GK_TRY(scr.alloc(&d_w0, nwin));
            GK_TRY(scr.alloc(&d_w1, nwin));
            GK_TRY(scr.alloc(&d_wo, nwin));
            GK_CUDA(ctx, cudaMemcpyAsync(d_wf, wf.data(), sizeof(int) * nwin, cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemcpyAsync(d_w0, w0.data(), sizeof(int64_t) * nwin, cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemcpyAsync(d_w1, w1.data(), sizeof(int64_t) * nwin, cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemcpyAsync(d_wo, wo.data(), sizeof(int64_t) * nwin, cudaMemcpyHostToDevice, st));
            uint64_t *klo, *khi;
            GK_TRY(scr.alloc(&klo, W));
            GK_TRY(scr.alloc(&khi, W));
            GK_COUNT();
            k_qalsh_gather<<<(unsigned)std::min<int64_t>(ceil_div(nwin, 8), (int64_t)ctx->num_sms * 16), 256, 0, st>>>(
                nwin, d_wf, d_w0, d_w1, d_wo, ids, n, x, ldx, d, a, klo, khi);
            GK_LAUNCH(ctx);
            GK_TRY(radix_sort_segments(ctx, scr, 1, W, &klo, &khi, nullptr, 96 + bit_length_u64((uint64_t)nwin),
                                       st));
            GK_COUNT();
            k_qalsh_put<<<grid_for(W, 256, ctx->num_sms), 256, 0, st>>>(W, klo, khi, d_wf, d_w0, d_wo, ids, n);
            GK_LAUNCH(ctx);
            // the pageable window tables above are read by the copies: keep
            // them until the stream got past them
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
    }
    GK_COUNT();
    k_qalsh_parts<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), m), 256, 0, st>>>(n, m, t, ids,
                                                                                              b->obj_bucket);
    GK_LAUNCH(ctx);
    uint64_t *bkey;
    GK_TRY(scr.alloc(&bkey, tot));
    GK_COUNT();
    k_qalsh_member_keys<<<grid_for(tot, 256, ctx->num_sms), 256, 0, st>>>(tot, n, b->obj_bucket, bkey, ids);
    GK_LAUNCH(ctx);
    GK_TRY(radix_sort_segments(ctx, scr, m, n, &bkey, nullptr, &ids, std::max(1, bit_length_u64((uint64_t)(t - 1))),
                               st));
    GK_COUNT();
    k_qalsh_boff<<<grid_for(b->NB + 1, 256, ctx->num_sms), 256, 0, st>>>(n, m, t, b->boff);
    GK_LAUNCH(ctx);
    return sort_err_check(ctx, st);
}
