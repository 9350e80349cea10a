// Alg. 1 (Sect. 3.1, homogeneous dense data): m QALSH projections
// s = a_f . x, each table sorted by (s, object id) and cut into t parts of
// sizes floor((j + 1) n / t) - floor(j n / t).
//
// The projections are computed with compensated FP32 arithmetic (Dot2, see
// k_qalsh_dot2) and each table is sorted by the double hi + lo.  With E a
// bound on |(hi + lo) - s| that holds for every object (s the pinned FP64
// dot product), the exact value tau at cut position p lies within E of the
// sorted value there (order statistics move by at most the largest
// perturbation).  So every object whose value is more than 2E below (above)
// the value at p is exactly before (after) the cut, and only the objects in
// the window [v_(p) - 2E, v_(p) + 2E] of the sorted order can change sides:
// their FP64 values are computed and each window (windows that overlap are
// merged) is re-sorted by (s, id).  Outside the windows the sorted position
// already gives the exact part.
#include <algorithm>

#include "internal.cuh"

namespace {

// order-preserving unsigned keys of IEEE values
__device__ __forceinline__ uint64_t f64_key(double v) {
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | (1ull << 63));
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

// ---- compensated projections ----------------------------------------------
// At large n the FP32 values are too coarse for the cuts: 10M values in a
// range of a few thousand are a few ulps apart, far inside the FP32 error
// bound, so every cut window would span whole tables.  This kernel computes
// each a_f . x_i with Dot2 (Ogita, Rump and Oishi; TwoProduct by FMA and
// TwoSum, coordinates in order): hi + lo is within gamma_d^2 sum|a_j x_j| of
// the exact dot product, so the windows shrink to the objects that are
// genuinely within ~1e-10 |a||x| of a cut.  Register tile 4 rows x 8
// functions per thread; x and a staged through shared memory in 32-wide
// k-chunks (cp.async, double buffered, 16-byte pieces XOR-swizzled by row).
constexpr int QD_T = 256, QD_RPT = 4, QD_FPT = 8, QD_KC = 32;

// |a_f| (FP32, sequential, times 1.0001: an upper bound)
__global__ void k_qalsh_anorm(const float *__restrict__ a, int F, int d, float *__restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    float s = 0.f;
    for (int j = 0; j < d; j++) s = fmaf(a[(int64_t)f * d + j], a[(int64_t)f * d + j], s);
    out[f] = sqrtf(s) * 1.0001f;
}

struct QDArgs {
    const float *x;
    int64_t ldx, n;
    int d, F, FPAD, FG, RG;
    const float *a;
    float *hi, *lo;      // n x F
    unsigned *xmax_bits; // max row-norm bound (float bits)
};

__device__ __forceinline__ void qd_term(float av, float xv, float &sh, float &sc) {
    const float p = __fmul_rn(av, xv);
    const float h = fmaf(av, xv, -p);  // exact product error
    const float s = __fadd_rn(sh, p);  // TwoSum(sh, p)
    const float z = __fsub_rn(s, sh);
    const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
    sh = s;
    sc = __fadd_rn(sc, __fadd_rn(er, h));
}

__global__ void __launch_bounds__(QD_T, 2) k_qalsh_dot2(QDArgs A) {
    extern __shared__ float sm[];
    const int TR = A.RG * QD_RPT, SR = TR + A.FPAD;
    float *st0 = sm, *st1 = sm + (size_t)SR * QD_KC;
    const int t = threadIdx.x, fg = t % A.FG, rg = t / A.FG;
    const bool active = t < A.FG * A.RG;
    const int64_t row0 = (int64_t)blockIdx.x * TR;
    const bool vec = ((A.ldx & 3) == 0) && ((A.d & 3) == 0) && (((uintptr_t)A.x & 15) == 0) &&
                     (((uintptr_t)A.a & 15) == 0);
    float sh[QD_RPT][QD_FPT], sc[QD_RPT][QD_FPT], xsq[QD_RPT];
#pragma unroll
    for (int r = 0; r < QD_RPT; r++) {
        xsq[r] = 0.f;
#pragma unroll
        for (int c = 0; c < QD_FPT; c++) sh[r][c] = sc[r][c] = 0.f;
    }
    auto stage = [&](float *buf, int k0) {
        for (int e = t; e < SR * 8; e += blockDim.x) {
            const int r = e >> 3, j = e & 7, k = k0 + 4 * j;
            const float *src;
            bool in;
            int sw;
            if (r < TR) {
                in = row0 + r < A.n;
                src = A.x + (row0 + r) * A.ldx + k;
                sw = r;
            } else {
                in = r - TR < A.F;
                src = A.a + (int64_t)(r - TR) * A.d + k;
                sw = r - TR;
            }
            float *dst = buf + r * QD_KC + 4 * (j ^ ((sw >> 3) & 7));
            const int nv = in ? max(0, min(4, A.d - k)) : 0;
            if (vec) {
                const uint32_t sa = (uint32_t)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(nv ? src : A.x),
                             "r"(nv * 4)
                             : "memory");
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++) dst[q] = q < nv ? src[q] : 0.f;
            }
        }
        if (vec) asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int nchunks = (A.d + QD_KC - 1) / QD_KC;
    stage(st0, 0);
    for (int ci = 0; ci < nchunks; ci++) {
        float *cur = (ci & 1) ? st1 : st0;
        if (ci + 1 < nchunks) {
            stage((ci & 1) ? st0 : st1, (ci + 1) * QD_KC);
            if (vec) asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else if (vec) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (active) {
            const float *xb = cur, *ab = cur + (size_t)TR * QD_KC;
            const int kmax = min(QD_KC, A.d - ci * QD_KC);
            for (int jb = 0; jb < (kmax + 3) / 4; jb++) {
                float4 xv[QD_RPT];
#pragma unroll
                for (int q = 0; q < QD_RPT; q++) {
                    const int r = rg * QD_RPT + q;
                    xv[q] = *reinterpret_cast<const float4 *>(xb + r * QD_KC + 4 * (jb ^ ((r >> 3) & 7)));
                    xsq[q] = fmaf(xv[q].x, xv[q].x, fmaf(xv[q].y, xv[q].y, fmaf(xv[q].z, xv[q].z,
                                                                                fmaf(xv[q].w, xv[q].w, xsq[q]))));
                }
#pragma unroll
                for (int c = 0; c < QD_FPT; c++) {
                    const int f = fg * QD_FPT + c;
                    const float4 av = *reinterpret_cast<const float4 *>(ab + f * QD_KC + 4 * (jb ^ ((f >> 3) & 7)));
#pragma unroll
                    for (int q = 0; q < QD_RPT; q++) {
                        qd_term(av.x, xv[q].x, sh[q][c], sc[q][c]);
                        qd_term(av.y, xv[q].y, sh[q][c], sc[q][c]);
                        qd_term(av.z, xv[q].z, sh[q][c], sc[q][c]);
                        qd_term(av.w, xv[q].w, sh[q][c], sc[q][c]);
                    }
                }
            }
        }
        __syncthreads();
    }
    float xm = 0.f;
    if (active) {
#pragma unroll
        for (int r = 0; r < QD_RPT; r++) {
            const int64_t row = row0 + rg * QD_RPT + r;
            if (row >= A.n) continue;
            xm = fmaxf(xm, sqrtf(xsq[r]) * 1.0001f);
#pragma unroll
            for (int c = 0; c < QD_FPT; c++) {
                const int f = fg * QD_FPT + c;
                if (f < A.F) {
                    A.hi[row * A.F + f] = sh[r][c];
                    A.lo[row * A.F + f] = sc[r][c];
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    if ((t & 31) == 0 && xm > 0.f) atomicMax(A.xmax_bits, __float_as_uint(xm));
}

// keys[f][i] = key of the double hi + lo of (i, f); ids[f][i] = i
__global__ void k_qalsh_keys2(int64_t n, int m, const float *__restrict__ hi, const float *__restrict__ lo,
                              uint64_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < m; f++) {
            const double v = __dadd_rn((double)hi[i * m + f], (double)lo[i * m + f]);
            keys[(int64_t)f * n + i] = f64_key(__dadd_rn(v, 0.0));
            ids[(int64_t)f * n + i] = (uint32_t)i;
        }
    }
}

__device__ __forceinline__ double key_f64(uint64_t k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}

// window of cut j (1 .. t-1) of table f in the compensated order: positions
// whose value is within 2.01 E of the value at floor(j n / t)
__global__ void k_qalsh_windows2(int64_t n, int m, int t, const uint64_t *__restrict__ keys,
                                 const float *__restrict__ anorm, const unsigned *__restrict__ xmax_bits, double cf,
                                 int64_t *__restrict__ q0, int64_t *__restrict__ q1) {
    const int64_t tot = (int64_t)m * (t - 1);
    const double xm = (double)__uint_as_float(*xmax_bits);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / (t - 1));
        const int64_t j = e % (t - 1) + 1;
        const uint64_t *kf = keys + (int64_t)f * n;
        const double v = key_f64(kf[j * n / t]);
        const double E = cf * (double)anorm[f] * xm;
        double lo = nextafter(__dsub_rn(v, 2.01 * E), -INFINITY), hi = nextafter(__dadd_rn(v, 2.01 * E), INFINITY);
        if (lo == 0.0) lo = -0.0;
        if (hi == 0.0) hi = 0.0;
        q0[e] = lower_key(kf, n, f64_key(lo), false);
        q1[e] = lower_key(kf, n, f64_key(hi), true);
    }
}

// one thread per list entry e (merged window w = the last with woff[w] <= e:
// table wf[w], position wq0[w] + e - woff[w]): the pinned FP64 dot product
// of the object there, keyed (window, FP64 value, id) for one sort of all
// windows.  Per entry, not per window: merged windows can span whole tables.
__global__ void k_qalsh_gather(int64_t W, int64_t nwin, const int *__restrict__ wf, const int64_t *__restrict__ wq0,
                               const int64_t *__restrict__ woff, const uint32_t *__restrict__ ids, int64_t n,
                               const float *__restrict__ x, int64_t ldx, int d, const float *__restrict__ a,
                               uint64_t *__restrict__ klo, uint64_t *__restrict__ khi) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < W; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nwin - 1;  // last window starting at or before e
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (woff[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int64_t w = lo;
        const int f = wf[w];
        const uint32_t id = ids[(int64_t)f * n + wq0[w] + (e - woff[w])];
        const float *xr = x + (int64_t)id * ldx;
        const float *af = a + (int64_t)f * d;
        double s = 0.0;
        for (int j = 0; j < d; j++) s = __dadd_rn(s, __dmul_rn((double)af[j], (double)xr[j]));
        const uint64_t k = f64_key(__dadd_rn(s, 0.0));  // -0 -> +0: equal values tie by id
        khi[e] = ((uint64_t)w << 32) | (k >> 32);
        klo[e] = (k << 32) | id;
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
    float *anorm, *lo;
    unsigned *xmax;
    GK_TRY(scr.alloc(&anorm, m));
    GK_TRY(scr.alloc(&xmax, 1));
    GK_CUDA(ctx, cudaMemsetAsync(xmax, 0, sizeof(unsigned), st));
    GK_COUNT();
    k_qalsh_anorm<<<(m + 127) / 128, 128, 0, st>>>(a, m, d, anorm);
    GK_LAUNCH(ctx);
    b->nb.assign(m, n > 0 ? t : 0);
    b->NB = n > 0 ? (int64_t)m * t : 0;
    b->key_bits_max = 64;
    GK_CUDA(ctx, cudaMallocAsync((void **)&b->boff, sizeof(int64_t) * (b->NB + 1), st));
    if (n == 0) {
        GK_CUDA(ctx, cudaMemsetAsync(b->boff, 0, sizeof(int64_t), st));
        return GEEK_OK;
    }
    const int64_t tot = n * m;
    GK_TRY(scr.alloc(&lo, tot));
    {
        QDArgs Q{};
        Q.x = x; Q.ldx = ldx; Q.n = n; Q.d = d; Q.F = m; Q.a = a;
        Q.FG = (m + QD_FPT - 1) / QD_FPT;
        Q.FPAD = Q.FG * QD_FPT;
        Q.RG = std::max(1, std::min(64, QD_T / Q.FG));
        Q.hi = (float *)b->codes;  // the handle's codes: FP32 bit patterns of hi
        Q.lo = lo;
        Q.xmax_bits = xmax;
        const int TR = Q.RG * QD_RPT;
        const int threads = (int)ceil_div(Q.FG * Q.RG, 32) * 32;
        const size_t smem = 2 * (size_t)QD_KC * (TR + Q.FPAD) * sizeof(float);
        if (smem > 200 * 1024) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "QALSH: projection tile too large");
        GK_CUDA(ctx, cudaFuncSetAttribute(k_qalsh_dot2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EvTimer tk(ctx, "kernel.project_dot2", st);
        tk.work = 2.0 * (double)n * (double)m * (double)d;
        GK_COUNT();
        k_qalsh_dot2<<<(unsigned)ceil_div(n, TR), threads, smem, st>>>(Q);
        GK_LAUNCH(ctx);
    }
    uint64_t *keys;
    GK_TRY(scr.alloc(&keys, tot));
    uint32_t *ids = b->members;  // the sorted order first, the members at the end
    GK_COUNT();
    k_qalsh_keys2<<<grid_for(n, 256, ctx->num_sms), 256, 0, st>>>(n, m, (const float *)b->codes, lo, keys, ids);
    GK_LAUNCH(ctx);
    {
        EvTimer tk(ctx, "hash.sort", st);
        GK_TRY(radix_sort_segments(ctx, scr, m, n, &keys, nullptr, &ids, 64, st));
    }
    if (t > 1) {
        const int64_t nc = (int64_t)m * (t - 1);
        int64_t *q0, *q1;
        GK_TRY(scr.alloc(&q0, nc));
        GK_TRY(scr.alloc(&q1, nc));
        // Dot2 against the exact value: gamma_d^2 <= 2.2 (2d)(d+1) 2^-48; the
        // double sum hi + lo and the FP64 reference: (d + 2) 2^-52
        const double cf = 2.2 * (2.0 * d) * (d + 1.0) * 3.552713678800501e-15 + (d + 2.0) * 2.220446049250313e-16;
        GK_COUNT();
        k_qalsh_windows2<<<grid_for(nc, 256, ctx->num_sms), 256, 0, st>>>(n, m, t, keys, anorm, xmax, cf, q0, q1);
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
            int64_t *d_w0, *d_wo;
            GK_TRY(scr.alloc(&d_wf, nwin));
            GK_TRY(scr.alloc(&d_w0, nwin));
            GK_TRY(scr.alloc(&d_wo, nwin));
            GK_CUDA(ctx, cudaMemcpyAsync(d_wf, wf.data(), sizeof(int) * nwin, cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemcpyAsync(d_w0, w0.data(), sizeof(int64_t) * nwin, cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemcpyAsync(d_wo, wo.data(), sizeof(int64_t) * nwin, cudaMemcpyHostToDevice, st));
            uint64_t *klo, *khi;
            GK_TRY(scr.alloc(&klo, W));
            GK_TRY(scr.alloc(&khi, W));
            GK_COUNT();
            k_qalsh_gather<<<grid_for(W, 256, ctx->num_sms), 256, 0, st>>>(W, nwin, d_wf, d_w0, d_wo, ids, n, x,
                                                                            ldx, d, a, klo, khi);
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
