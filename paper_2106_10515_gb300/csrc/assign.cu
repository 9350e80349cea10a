// Central vectors and one-pass data assignment (Sect. 3.3, Eq. 1).
//
// Dense assignment evaluates d'_j = |c_j|^2 - 2 x.c_j (the row-constant
// |x|^2 dropped) for every centre in a fast precision, keeps the best and
// second-best value per object, and decides the argmin in FP64 only for
// objects whose gap is within the rigorous error window.  The FP64 decision
// reproduces the reference distance exactly: sum_t ((double)x_t - c_t)^2 in t
// order, each operation rounded to nearest, no fused multiply-add; ties go
// to the smallest centre index.
#include <cfloat>

#include "internal.cuh"

namespace {

constexpr int AS_TR = 128;   // rows per block
constexpr int AS_TC = 64;    // centres per tile
constexpr int AS_KC = 32;    // d-chunk of the centre tile
constexpr int AS_RPT = 8;    // rows per thread
constexpr int AS_CPT = 4;    // centres per thread
constexpr int AS_MAXD = 256; // X tile resident in shared memory

// FP64 reference distance of the pinned definition.
__device__ __forceinline__ double ref_dist(const float *__restrict__ x, const double *__restrict__ c, int d) {
    double D = 0.0;
    for (int t = 0; t < d; t++) {
        const double e = __dsub_rn((double)x[t], c[t]);
        D = __dadd_rn(D, __dmul_rn(e, e));
    }
    return D;
}

// Rigorous half-window of the FP32 path for one object (see the proof in
// the file header): (2 gamma_d + 4u)|x| cmax + 2u cmax^2 for the fast value,
// plus the FP64 reference's own error (d+3) 2^-53 (|x| + cmax)^2, times 1.01.
__device__ __forceinline__ float window_fp32(float xn, float cmax, int d) {
    const float u = 5.9604645e-8f;
    const float gam = (float)d * u / (1.f - (float)d * u);
    const float e32 = (2.f * gam + 4.f * u) * xn * cmax + 2.f * u * cmax * cmax;
    const float s = xn + cmax;
    const float e64 = (float)(d + 3) * 1.1102230e-16f * s * s;
    return 1.01f * (e32 + e64) + 1e-30f;
}

struct Best {
    float b1, b2;
    int i1;
};

__device__ __forceinline__ void best_push(Best &B, float v, int j) {
    if (v < B.b1) {
        B.b2 = B.b1;
        B.b1 = v;
        B.i1 = j;
    } else {
        B.b2 = fminf(B.b2, v);
    }
}

__device__ __forceinline__ Best best_merge(Best a, Best b) {
    Best r;
    const bool take_b = b.b1 < a.b1 || (b.b1 == a.b1 && b.i1 < a.i1);
    r.b1 = take_b ? b.b1 : a.b1;
    r.i1 = take_b ? b.i1 : a.i1;
    r.b2 = fminf(fminf(a.b2, b.b2), take_b ? a.b1 : b.b1);
    return r;
}

// FP32 SIMT assignment: block = 128 rows, all centres streamed in tiles of
// 64; 256 threads = 16 row groups (8 rows) x 16 centre groups (4 centres).
__global__ void __launch_bounds__(256) k_assign_fp32(const float *__restrict__ x, int64_t ldx, int64_t n,
                                                     int d, const float *__restrict__ c32,
                                                     const float *__restrict__ cn, int64_t k, float cmax,
                                                     int32_t *__restrict__ labels,
                                                     int32_t *__restrict__ flag_rows,
                                                     unsigned long long *__restrict__ n_flag) {
    extern __shared__ float sm[];
    float *xs = sm;                         // [d][AS_TR]
    float *cs = sm + (size_t)d * AS_TR;     // [AS_KC][AS_TC]
    __shared__ float cns[AS_TC];
    const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * AS_TR;
    for (int e = t; e < AS_TR * d; e += 256) {
        const int r = e / d, kk = e % d;
        const int64_t row = row0 + r;
        xs[kk * AS_TR + r] = row < n ? x[row * ldx + kk] : 0.f;
    }
    Best B[AS_RPT];
#pragma unroll
    for (int r = 0; r < AS_RPT; r++) B[r] = Best{FLT_MAX, FLT_MAX, 0x7FFFFFFF};
    for (int64_t j0 = 0; j0 < k; j0 += AS_TC) {
        float acc[AS_RPT][AS_CPT];
#pragma unroll
        for (int r = 0; r < AS_RPT; r++)
#pragma unroll
            for (int c = 0; c < AS_CPT; c++) acc[r][c] = 0.f;
        for (int k0 = 0; k0 < d; k0 += AS_KC) {
            __syncthreads();
            for (int e = t; e < AS_TC * AS_KC; e += 256) {
                const int c = e / AS_KC, kk = e % AS_KC;
                const int64_t j = j0 + c;
                cs[kk * AS_TC + c] = (j < k && k0 + kk < d) ? c32[j * d + k0 + kk] : 0.f;
            }
            if (k0 == 0 && t < AS_TC) cns[t] = j0 + t < k ? cn[j0 + t] : FLT_MAX;
            __syncthreads();
            const int kmax = min(AS_KC, d - k0);
            for (int kk = 0; kk < kmax; kk++) {
                const float4 x0 = *reinterpret_cast<const float4 *>(&xs[(k0 + kk) * AS_TR + rg * AS_RPT]);
                const float4 x1 = *reinterpret_cast<const float4 *>(&xs[(k0 + kk) * AS_TR + rg * AS_RPT + 4]);
                const float4 cv = *reinterpret_cast<const float4 *>(&cs[kk * AS_TC + cg * AS_CPT]);
                const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                for (int r = 0; r < AS_RPT; r++)
#pragma unroll
                    for (int c = 0; c < AS_CPT; c++) acc[r][c] = fmaf(xv[r], cc[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int c = 0; c < AS_CPT; c++) {
            const int64_t j = j0 + cg * AS_CPT + c;
            if (j >= k) continue;
            const float cnj = cns[cg * AS_CPT + c];
#pragma unroll
            for (int r = 0; r < AS_RPT; r++) best_push(B[r], fmaf(-2.f, acc[r][c], cnj), (int)j);
        }
    }
    // merge the 16 centre groups of each row group (lanes of one half-warp)
#pragma unroll
    for (int r = 0; r < AS_RPT; r++) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            Best o_;
            o_.b1 = __shfl_xor_sync(0xffffffffu, B[r].b1, o);
            o_.b2 = __shfl_xor_sync(0xffffffffu, B[r].b2, o);
            o_.i1 = __shfl_xor_sync(0xffffffffu, B[r].i1, o);
            B[r] = best_merge(B[r], o_);
        }
    }
    if (cg == 0) {
#pragma unroll
        for (int r = 0; r < AS_RPT; r++) {
            const int64_t row = row0 + rg * AS_RPT + r;
            if (row >= n) continue;
            float xs2 = 0.f;
            for (int kk = 0; kk < d; kk++) {
                const float v = xs[kk * AS_TR + rg * AS_RPT + r];
                xs2 = fmaf(v, v, xs2);
            }
            const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
            const float W = 2.f * window_fp32(xn, cmax, d);
            // no finite value (non-finite input): undecided here, FP64 decides
            const bool valid = B[r].i1 != 0x7FFFFFFF;
            labels[row] = valid ? B[r].i1 : -1;
            const bool sure = valid && (k == 1 || (B[r].b2 - B[r].b1 > W * (1.f + 1e-6f)));
            if (!sure) {
                const unsigned long long q = atomicAdd(n_flag, 1ull);
                flag_rows[q] = (int32_t)row;
            }
        }
    }
}

// Exact decision for one flagged object: FP32 filter over all centres, then
// the FP64 reference distance for every centre inside the window.  Flag
// entries are global rows; instance i owns rows [row_off[i], row_off[i+1]).
__global__ void __launch_bounds__(256) k_assign_recheck(const RInst *__restrict__ R,
                                                        const int64_t *__restrict__ row_off, int count,
                                                        const int32_t *__restrict__ flag_rows,
                                                        const unsigned long long *__restrict__ n_flag) {
    extern __shared__ float xr[];  // d floats
    __shared__ float red_f[256];
    __shared__ double red_d[256];
    __shared__ int red_i[256];
    const int t = threadIdx.x;
    const int64_t nf = (int64_t)*n_flag;
    for (int64_t q = blockIdx.x; q < nf; q += gridDim.x) {
        const int64_t grow = flag_rows[q];
        const RInst &I = R[find_inst(row_off, count, grow)];
        const int64_t row = grow - I.row_base;
        const int d = I.d;
        const int64_t k = I.k;
        const float *c32 = I.c32, *cn = I.cn;
        const float cmax = __uint_as_float(*I.cmax_bits);
        __syncthreads();
        for (int kk = t; kk < d; kk += 256) xr[kk] = I.x[row * I.ldx + kk];
        __syncthreads();
        float xs2 = 0.f;
        for (int kk = 0; kk < d; kk++) xs2 = fmaf(xr[kk], xr[kk], xs2);
        const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
        float m = FLT_MAX;
        for (int64_t j = t; j < k; j += 256) {
            float dot = 0.f;
            for (int kk = 0; kk < d; kk++) dot = fmaf(xr[kk], c32[j * d + kk], dot);
            m = fminf(m, fmaf(-2.f, dot, cn[j]));
        }
        red_f[t] = m;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (t < o) red_f[t] = fminf(red_f[t], red_f[t + o]);
            __syncthreads();
        }
        const float lim = red_f[0] + 2.f * window_fp32(xn, cmax, d) * (1.f + 1e-6f);
        double bD = DBL_MAX;
        int bj = 0x7FFFFFFF;
        for (int64_t j = t; j < k; j += 256) {
            float dot = 0.f;
            for (int kk = 0; kk < d; kk++) dot = fmaf(xr[kk], c32[j * d + kk], dot);
            if (fmaf(-2.f, dot, cn[j]) <= lim) {
                const double D = ref_dist(xr, I.c64 + j * d, d);
                if (D < bD || (D == bD && (int)j < bj)) {
                    bD = D;
                    bj = (int)j;
                }
            }
        }
        red_d[t] = bD;
        red_i[t] = bj;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (t < o) {
                const double D2 = red_d[t + o];
                const int j2 = red_i[t + o];
                if (D2 < red_d[t] || (D2 == red_d[t] && j2 < red_i[t])) {
                    red_d[t] = D2;
                    red_i[t] = j2;
                }
            }
            __syncthreads();
        }
        // no candidate with a distance below +inf (non-finite input): -1,
        // as the reference argmin that never improves on +inf
        if (t == 0) I.labels[row] = red_i[0] == 0x7FFFFFFF ? -1 : red_i[0];
    }
}

// centre preparation: FP32 copy, |c|^2 (FP64 then rounded), max |c|;
// thread per global centre e of instance find_inst(k_off, e)
__global__ void k_centre_prep(const CInst *__restrict__ C, const int64_t *__restrict__ k_off, int count,
                              int64_t ktot) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ktot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const CInst &I = C[find_inst(k_off, count, e)];
        const int64_t j = e - I.k_base;
        const int d = I.d;
        double s = 0.0;
        for (int t = 0; t < d; t++) {
            const double v = I.c64[j * d + t];
            I.c32[j * d + t] = (float)v;
            s += v * v;
        }
        I.cn[j] = (float)s;
        const float nrm = (float)sqrt(s) * (1.f + 1e-6f);
        atomicMax(I.cmax_bits, __float_as_uint(nrm));  // non-negative floats order as uints
    }
}

// double-float split of the FP64 centres: c = hi + lo with hi = (float)c
__global__ void k_centre_split(const double *__restrict__ c64, int64_t kd, float *__restrict__ hi,
                               float *__restrict__ lo) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x) {
        const double c = c64[e];
        const float h = (float)c;
        hi[e] = h;
        lo[e] = (float)(c - (double)h);
    }
}

// per-object distance to its centre, warp per object, lanes over
// coordinates: diff = (x - c_hi) - c_lo, squares accumulated in FP32; block
// partial sums (FP64) and maxima, reduced on one block in a fixed order
__global__ void __launch_bounds__(256) k_assign_stats(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                                      const float *__restrict__ chi, const float *__restrict__ clo,
                                                      int64_t k, const int32_t *__restrict__ labels,
                                                      double *__restrict__ part_sum, float *__restrict__ part_max) {
    __shared__ double ss[8];
    __shared__ float sm_[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double s = 0.0;
    float mx = 0.f;
    for (int64_t i = warp; i < n; i += nw) {
        const int j = labels[i];
        if (j < 0 || j >= k) continue;  // uniform across the warp
        const float *xr = x + i * ldx;
        const float *h = chi + (int64_t)j * d;
        const float *l = clo + (int64_t)j * d;
        float D = 0.f;
        for (int t = lane; t < d; t += 32) {
            const float e = (xr[t] - h[t]) - l[t];
            D = fmaf(e, e, D);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) D += __shfl_xor_sync(0xffffffffu, D, o);
        s += (double)D;
        mx = fmaxf(mx, D);
    }
    if (lane == 0) {
        ss[wib] = s;
        sm_[wib] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        float m = 0.f;
        for (int w = 0; w < 8; w++) {
            a += ss[w];
            m = fmaxf(m, sm_[w]);
        }
        part_sum[blockIdx.x] = a;
        part_max[blockIdx.x] = m;
    }
}

__global__ void k_stats_final(const double *__restrict__ ps, const float *__restrict__ pm, int nb,
                              double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        float m = 0.f;
        for (int i = 0; i < nb; i++) {
            s += ps[i];
            m = fmaxf(m, pm[i]);
        }
        out[0] = s;
        out[1] = sqrt((double)m);
    }
}

// centroid coordinate t of the seed with members sids[s0 .. s1) (ascending
// ids, rows x + (id - row_base) * ldx): FP64 sum in member order, one IEEE
// division by the count
__device__ __forceinline__ double centroid_coord(const float *__restrict__ x, int64_t ldx, int64_t row_base,
                                                 const int32_t *__restrict__ sids, int64_t s0, int64_t s1, int t) {
    double s = 0.0;
    for (int64_t p = s0; p < s1; p++) s = __dadd_rn(s, (double)x[((int64_t)sids[p] - row_base) * ldx + t]);
    return __ddiv_rn(s, (double)(s1 - s0));
}

// centroid of each seed; one thread per (seed, coordinate)
__global__ void k_centroids(const float *__restrict__ x, int64_t ldx, int d, int64_t k,
                            const int64_t *__restrict__ soff, const int32_t *__restrict__ sids,
                            double *__restrict__ c) {
    const int64_t total = k * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / d;
        const int t = (int)(e % d);
        c[e] = centroid_coord(x, ldx, 0, sids, soff[j], soff[j + 1], t);
    }
}

// batched: thread per (global seed, coordinate < dmax); instance i owns
// seeds [seed_inst_off[i], seed_inst_off[i + 1])
__global__ void k_centroids_batch(const CenInst *__restrict__ C, const int64_t *__restrict__ seed_inst_off,
                                  int count, int64_t ktot, int dmax, const int64_t *__restrict__ soff,
                                  const int32_t *__restrict__ sids) {
    const int64_t total = ktot * dmax;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / dmax;
        const int t = (int)(e % dmax);
        const CenInst &I = C[find_inst(seed_inst_off, count, s)];
        if (t >= I.d) continue;
        I.c[(s - I.seed_base) * I.d + t] = centroid_coord(I.x, I.ldx, I.row_base, sids, soff[s], soff[s + 1], t);
    }
}

// batched SSE / radius partials: block per 128-row unit (instance, tile),
// warp per row, squares of (x - c_hi) - c_lo accumulated in FP32
__global__ void __launch_bounds__(256) k_assign_stats_batch(const SInst *__restrict__ S, const int2 *__restrict__ units,
                                                            int64_t nunits, double *__restrict__ part_sum,
                                                            float *__restrict__ part_max) {
    __shared__ double ss[8];
    __shared__ float sm_[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int2 un = units[u];
        const SInst &I = S[un.x];
        double s = 0.0;
        float mx = 0.f;
        for (int r = wib; r < 128; r += 8) {
            const int64_t i = (int64_t)un.y * 128 + r;
            if (i >= I.n) break;
            const int j = I.labels[i];
            if (j < 0 || j >= I.k) continue;  // uniform across the warp
            const float *xr = I.x + i * I.ldx;
            const float *h = I.chi + (int64_t)j * I.d;
            const float *l = I.clo + (int64_t)j * I.d;
            float D = 0.f;
            for (int t = lane; t < I.d; t += 32) {
                const float e = (xr[t] - h[t]) - l[t];
                D = fmaf(e, e, D);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) D += __shfl_xor_sync(0xffffffffu, D, o);
            s += (double)D;
            mx = fmaxf(mx, D);
        }
        __syncthreads();
        if (lane == 0) {
            ss[wib] = s;
            sm_[wib] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            float m = 0.f;
            for (int w = 0; w < 8; w++) {
                a += ss[w];
                m = fmaxf(m, sm_[w]);
            }
            part_sum[u] = a;
            part_max[u] = m;
        }
    }
}

// per instance: its units' partials in unit order (deterministic)
__global__ void k_stats_final_batch(const double *__restrict__ ps, const float *__restrict__ pm,
                                    const int64_t *__restrict__ unit_off, int count, double *__restrict__ sse,
                                    double *__restrict__ rmax) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        float m = 0.f;
        for (int64_t u = unit_off[i]; u < unit_off[i + 1]; u++) {
            s += ps[u];
            m = fmaxf(m, pm[u]);
        }
        sse[i] = s;
        rmax[i] = sqrt((double)m);
    }
}

__global__ void k_fill_labels(int32_t *l, int64_t n, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        l[i] = v;
}

}  // namespace

geek_status centroids_from_seeds(geek_ctx *ctx, const float *x, int64_t ldx, int d, const silk_seeds *s,
                                 double *centres, cudaStream_t st) {
    if (s->k == 0) return GEEK_OK;
    GK_COUNT();
    k_centroids<<<grid_for(s->k * d, 256, ctx->num_sms), 256, 0, st>>>(x, ldx, d, s->k, s->off, s->ids, centres);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status assign_dense_centres(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                                 const double *centres, int64_t k, int precision, int32_t *labels,
                                 geek_assign_stats *stats, cudaStream_t st) {
    if (stats) *stats = geek_assign_stats{0.0, 0.0, k, 0};
    if (n == 0) return GEEK_OK;
    if (k == 0) {
        GK_COUNT();
        k_fill_labels<<<grid_for(n, 256, ctx->num_sms), 256, 0, st>>>(labels, n, -1);
        GK_LAUNCH(ctx);
        return GEEK_OK;
    }
    if (d > AS_MAXD) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "dense assignment supports d <= %d", AS_MAXD);
    if (precision != GEEK_PREC_FP32 && precision != GEEK_PREC_BF16)
        return set_error(ctx, GEEK_ERR_INVALID, "bad precision");
    float *c32, *cn;
    unsigned *cmax_bits;
    GK_TRY(scr.alloc(&c32, (size_t)k * d));
    GK_TRY(scr.alloc(&cn, k));
    GK_TRY(scr.alloc(&cmax_bits, 1));
    GK_CUDA(ctx, cudaMemsetAsync(cmax_bits, 0, sizeof(unsigned), st));
    // one-instance tables for the instance-driven kernels
    CInst *ci;
    RInst *ri;
    int64_t *koff, *roff;
    GK_TRY(scr.alloc(&ci, 1));
    GK_TRY(scr.alloc(&ri, 1));
    GK_TRY(scr.alloc(&koff, 2));
    GK_TRY(scr.alloc(&roff, 2));
    {
        const CInst hc{centres, c32, cn, cmax_bits, d, 0};
        const RInst hr{x, ldx, d, c32, cn, centres, k, cmax_bits, labels, 0};
        const int64_t hk[2] = {0, k}, hn[2] = {0, n};
        GK_CUDA(ctx, cudaMemcpyAsync(ci, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaMemcpyAsync(ri, &hr, sizeof hr, cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaMemcpyAsync(koff, hk, sizeof hk, cudaMemcpyHostToDevice, st));
        GK_CUDA(ctx, cudaMemcpyAsync(roff, hn, sizeof hn, cudaMemcpyHostToDevice, st));
    }
    GK_COUNT();
    k_centre_prep<<<grid_for(k, 128, ctx->num_sms), 128, 0, st>>>(ci, koff, 1, k);
    GK_LAUNCH(ctx);
    unsigned h_bits = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_bits, cmax_bits, sizeof h_bits, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    float cmax;
    memcpy(&cmax, &h_bits, sizeof cmax);
    int32_t *flag_rows;
    unsigned long long *n_flag;
    GK_TRY(scr.alloc(&flag_rows, n));
    GK_TRY(scr.alloc(&n_flag, 1));
    GK_CUDA(ctx, cudaMemsetAsync(n_flag, 0, sizeof(unsigned long long), st));
    if (precision == GEEK_PREC_BF16) {
        GK_TRY(assign_tc_bf16(ctx, scr, x, ldx, n, d, centres, k, labels, flag_rows, n_flag, st));
    } else {
        const size_t smem = (size_t)d * AS_TR * sizeof(float) + (size_t)AS_KC * AS_TC * sizeof(float);
        GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EvTimer tk(ctx, "kernel.assign_fp32", st);
        tk.work = 2.0 * (double)n * (double)k * (double)d;
        GK_COUNT();
        k_assign_fp32<<<(unsigned)ceil_div(n, AS_TR), 256, smem, st>>>(x, ldx, n, d, c32, cn, k, cmax, labels,
                                                                         flag_rows, n_flag);
        GK_LAUNCH(ctx);
    }
    unsigned long long h_flag = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_flag, n_flag, sizeof h_flag, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_flag) {
        const int blocks = (int)std::min<unsigned long long>(h_flag, (unsigned long long)ctx->num_sms * 8);
        EvTimer tk(ctx, "kernel.assign_recheck", st);
        GK_COUNT();
        k_assign_recheck<<<blocks, 256, d * sizeof(float), st>>>(ri, roff, 1, flag_rows, n_flag);
        GK_LAUNCH(ctx);
    }
    if (stats) {
        const int nb = grid_for(n, 256, ctx->num_sms);
        double *ps, *out;
        float *pm;
        GK_TRY(scr.alloc(&ps, nb));
        GK_TRY(scr.alloc(&pm, nb));
        GK_TRY(scr.alloc(&out, 2));
        float *chi, *clo;
        GK_TRY(scr.alloc(&chi, (size_t)k * d));
        GK_TRY(scr.alloc(&clo, (size_t)k * d));
        GK_COUNT();
        k_centre_split<<<grid_for(k * d, 256, ctx->num_sms), 256, 0, st>>>(centres, k * d, chi, clo);
        GK_COUNT();
        k_assign_stats<<<nb, 256, 0, st>>>(x, ldx, n, d, chi, clo, k, labels, ps, pm);
        GK_COUNT();
        k_stats_final<<<1, 32, 0, st>>>(ps, pm, nb, out);
        GK_LAUNCH(ctx);
        double h[2];
        GK_CUDA(ctx, cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        stats->sse = h[0];
        stats->radius_max = h[1];
        stats->k = k;
        stats->n_recheck_rows = (int64_t)h_flag;
    }
    return GEEK_OK;
}

geek_status centroids_batch(geek_ctx *ctx, const CenInst *C, const int64_t *seed_inst_off, int count, int64_t ktot,
                            int dmax, const int64_t *soff, const int32_t *sids, cudaStream_t st) {
    if (ktot == 0) return GEEK_OK;
    GK_COUNT();
    k_centroids_batch<<<grid_for(ktot * dmax, 256, ctx->num_sms), 256, 0, st>>>(C, seed_inst_off, count, ktot, dmax,
                                                                              soff, sids);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status centre_prep_batch(geek_ctx *ctx, const CInst *C, const int64_t *k_off, int count, int64_t ktot,
                              cudaStream_t st) {
    if (ktot == 0) return GEEK_OK;
    GK_COUNT();
    k_centre_prep<<<grid_for(ktot, 128, ctx->num_sms), 128, 0, st>>>(C, k_off, count, ktot);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status recheck_batch(geek_ctx *ctx, const RInst *R, const int64_t *row_off, int count, int dmax,
                          const int32_t *flag_rows, const unsigned long long *n_flag, cudaStream_t st) {
    EvTimer tk(ctx, "kernel.assign_recheck", st);
    GK_COUNT();
    k_assign_recheck<<<ctx->num_sms * 8, 256, dmax * sizeof(float), st>>>(R, row_off, count, flag_rows, n_flag);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status centre_split(geek_ctx *ctx, const double *c64, int64_t total, float *chi, float *clo, cudaStream_t st) {
    if (total == 0) return GEEK_OK;
    GK_COUNT();
    k_centre_split<<<grid_for(total, 256, ctx->num_sms), 256, 0, st>>>(c64, total, chi, clo);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status stats_batch(geek_ctx *ctx, const SInst *S, const int2 *units, int64_t nunits, const int64_t *unit_off,
                        int count, double *part_sum, float *part_max, double *sse, double *rmax, cudaStream_t st) {
    if (nunits > 0) {
        GK_COUNT();
        k_assign_stats_batch<<<(int)std::min<int64_t>(nunits, (int64_t)ctx->num_sms * 16), 256, 0, st>>>(
            S, units, nunits, part_sum, part_max);
    }
    GK_COUNT();
    k_stats_final_batch<<<(count + 127) / 128, 128, 0, st>>>(part_sum, part_max, unit_off, count, sse, rmax);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status fill_labels(geek_ctx *ctx, int32_t *labels, int64_t n, int32_t v, cudaStream_t st) {
    if (n == 0) return GEEK_OK;
    GK_COUNT();
    k_fill_labels<<<grid_for(n, 256, ctx->num_sms), 256, 0, st>>>(labels, n, v);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}
