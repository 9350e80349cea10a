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
#include <type_traits>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int AS_TR = 128;   // rows per block
constexpr int AS_TC = 64;    // centres per tile
constexpr int AS_KC = 32;    // d-chunk of the centre tile
constexpr int AS_RPT = 8;    // rows per thread
constexpr int AS_CPT = 4;    // centres per thread
constexpr int AS_MAXD = 256; // X tile resident in shared memory

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
// GATHER = false: blocks walk the row tiles of the one data set A.
// GATHER = true: blocks walk units of up to 128 flagged rows of one instance
// (unit u: instance unit_inst[u], global rows grows[unit_start[u] ..
// + unit_cnt[u]]); the instance's data replace A's, uncertain rows are
// appended (as global rows) to A.flag_rows.
struct FArgs {
    const float *x;
    int64_t ldx, n;
    int d;
    const float *c32, *cn;
    int64_t k;
    float cmax;
    int32_t *labels;
    int32_t *flag_rows;
    float *flag_m;  // may be null: the row's smallest fast value, beside flag_rows
    unsigned long long *n_flag;
    int64_t ntiles;
};
struct GatherUnits {
    const RInst *R;
    const int32_t *grows;
    const int *unit_inst;
    const int64_t *unit_start;
    const int *unit_cnt;
    const int *n_units;
};

template <bool GATHER>
__global__ void __launch_bounds__(256) k_assign_fp32(FArgs A, GatherUnits U) {
    extern __shared__ float sm[];
    __shared__ float cns[AS_TC];
    __shared__ int64_t s_rows[AS_TR];
    const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
    const int64_t nunits = GATHER ? (int64_t)*U.n_units : A.ntiles;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        int64_t row0 = u * AS_TR;
        int nrows = (int)min((int64_t)AS_TR, A.n - row0);
        int64_t rbase = 0;
        if (GATHER) {
            const RInst &I = U.R[U.unit_inst[u]];
            A.x = I.x;
            A.ldx = I.ldx;
            A.d = I.d;
            A.c32 = I.c32;
            A.cn = I.cn;
            A.k = I.k;
            A.cmax = __uint_as_float(*I.cmax_bits);
            A.labels = I.labels;
            rbase = I.row_base;
            nrows = U.unit_cnt[u];
            __syncthreads();  // s_rows of the previous unit fully used
            if (t < nrows) s_rows[t] = (int64_t)U.grows[U.unit_start[u] + t] - rbase;
            __syncthreads();
        }
        const int d = A.d;
        const int64_t k = A.k;
        float *xs = sm;                         // [d][AS_TR]
        float *cs = sm + (size_t)d * AS_TR;     // [AS_KC][AS_TC]
        __syncthreads();
        for (int e = t; e < AS_TR * d; e += 256) {
            const int r = e / d, kk = e % d;
            float v = 0.f;
            if (r < nrows) v = A.x[(GATHER ? s_rows[r] : row0 + r) * A.ldx + kk];
            xs[kk * AS_TR + r] = v;
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
                    cs[kk * AS_TC + c] = (j < k && k0 + kk < d) ? A.c32[j * d + k0 + kk] : 0.f;
                }
                if (k0 == 0 && t < AS_TC) cns[t] = j0 + t < k ? A.cn[j0 + t] : FLT_MAX;
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
                const int rr = rg * AS_RPT + r;
                if (rr >= nrows) continue;
                const int64_t row = GATHER ? s_rows[rr] : row0 + rr;
                float xs2 = 0.f;
                for (int kk = 0; kk < d; kk++) {
                    const float v = xs[kk * AS_TR + rr];
                    xs2 = fmaf(v, v, xs2);
                }
                const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
                const float W = 2.f * window_fp32(xn, A.cmax, d);
                // no finite value (non-finite input): undecided here, FP64 decides
                const bool valid = B[r].i1 != 0x7FFFFFFF;
                A.labels[row] = valid ? B[r].i1 : -1;
                const bool sure = valid && (k == 1 || (B[r].b2 - B[r].b1 > W * (1.f + 1e-6f)));
                if (!sure) {
                    const unsigned long long q = atomicAdd(A.n_flag, 1ull);
                    A.flag_rows[q] = (int32_t)(rbase + row);
                    if (A.flag_m) A.flag_m[q] = valid ? B[r].b1 : __int_as_float(0x7fc00000);
                }
            }
        }
    }
}

// The tiled FP64 decision of the rows the FP32 refine leaves uncertain: the
// centres streamed through shared memory in tiles, the FP32 fast value of
// every (row, centre) pair in registers.  A pair whose fast value lies within
// the row's window lim = m + 2W (m: the row's smallest fast value, from the
// refine pass, in mrow[global row]) gets the FP64 reference distance, read
// from the row in shared memory; the row's label is the smallest reference
// distance, ties to the smaller index (-1 when no value is finite).
//
// The FP64 distances are a chain of d dependent adds each, and the FP64 pipe
// issues one warp-wide operation about every 19 cycles per SM: computed by
// the thread that found the pair, one active lane would pay for a whole
// warp.  So the tile's pairs go to a shared-memory queue and the block takes
// them a lane each (in rounds of at most DQ_CAP pairs); each row's best is
// kept in shared memory as the smallest D (an atomic minimum on its bits: D
// >= 0, so the bit order is the value order), then the smallest index among
// the pairs that reach it.
constexpr int DQ_CAP = 2048;
constexpr size_t DQ_BYTES = (size_t)DQ_CAP * (sizeof(double) + sizeof(uint16_t));

// exact FP32 -> FP64 widening in integer operations (normal, subnormal, zero,
// infinity; a NaN stays a NaN): keeps the conversion off the FP64 pipe
__device__ __forceinline__ double widen_f32(float v) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t sg = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    // subnormal: m = 1.f x 2^(p - 23) with p the top set bit, value m 2^-149
    const int sh = __clz((int)m) - 8;  // brings the top bit of m to bit 23
    const uint32_t ms = (m << (sh & 31)) & 0x7FFFFFu;
    const uint32_t es = (uint32_t)(1023 - 126 - sh);
    uint32_t hi, lo;
    if (e == 0u) {
        hi = m == 0u ? sg : (sg | (es << 20) | (ms >> 3));
        lo = m == 0u ? 0u : (ms << 29);
    } else {
        const uint32_t ed = e == 0xFFu ? 0x7FFu : e + 896u;
        hi = sg | (ed << 20) | (m >> 3);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double ref_dist_strided(const float *x, int stride, const double *__restrict__ c, int d) {
    double D = 0.0;
    for (int t = 0; t < d; t++) {
        const double e = __dsub_rn(widen_f32(x[t * stride]), c[t]);
        D = __dadd_rn(D, __dmul_rn(e, e));
    }
    return D;
}

__global__ void __launch_bounds__(256) k_assign_decide64(GatherUnits U, const float *__restrict__ mrow) {
    extern __shared__ float sm[];
    __shared__ float cns[AS_TC];
    __shared__ int64_t s_rows[AS_TR];
    __shared__ unsigned long long sbD[AS_TR], prevD[AS_TR];
    __shared__ int sbJ[AS_TR], tJ[AS_TR];
    __shared__ int s_qn;
    constexpr unsigned long long DINF = 0x7FF0000000000000ull;  // above every finite D
    const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
    const int64_t nunits = (int64_t)*U.n_units;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const RInst &I = U.R[U.unit_inst[u]];
        const int d = I.d;
        const int64_t k = I.k;
        const int64_t rbase = I.row_base;
        const int nrows = U.unit_cnt[u];
        __syncthreads();  // s_rows and xs of the previous unit fully used
        if (t < nrows) s_rows[t] = (int64_t)U.grows[U.unit_start[u] + t] - rbase;
        if (t < AS_TR) {
            sbD[t] = DINF;
            prevD[t] = DINF;
            sbJ[t] = 0x7FFFFFFF;
            tJ[t] = 0x7FFFFFFF;
        }
        if (t == 0) s_qn = 0;
        __syncthreads();
        float *xs = sm;                      // [d][AS_TR]
        float *cs = sm + (size_t)d * AS_TR;  // [AS_KC][AS_TC]
        double *qd = reinterpret_cast<double *>(cs + AS_KC * AS_TC);  // [DQ_CAP]
        uint16_t *qi = reinterpret_cast<uint16_t *>(qd + DQ_CAP);     // [DQ_CAP]: row * AS_TC + column
        for (int e = t; e < AS_TR * d; e += 256) {
            const int r = e / d, kk = e % d;
            xs[kk * AS_TR + r] = r < nrows ? I.x[s_rows[r] * I.ldx + kk] : 0.f;
        }
        __syncthreads();
        const float cmax = __uint_as_float(*I.cmax_bits);
        float lim[AS_RPT];
#pragma unroll
        for (int r = 0; r < AS_RPT; r++) {
            const int rr = rg * AS_RPT + r;
            float xs2 = 0.f;
            for (int kk = 0; kk < d; kk++) xs2 = fmaf(xs[kk * AS_TR + rr], xs[kk * AS_TR + rr], xs2);
            const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
            const float m = rr < nrows ? mrow[rbase + s_rows[rr]] : __int_as_float(0x7fc00000);
            lim[r] = m + 2.f * window_fp32(xn, cmax, d) * (1.f + 1e-6f);
        }
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
                    cs[kk * AS_TC + c] = (j < k && k0 + kk < d) ? I.c32[j * d + k0 + kk] : 0.f;
                }
                if (k0 == 0 && t < AS_TC) cns[t] = j0 + t < k ? I.cn[j0 + t] : FLT_MAX;
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
            // this thread's pairs inside the window: bit r * AS_CPT + c
            uint32_t pend = 0;
#pragma unroll
            for (int c = 0; c < AS_CPT; c++) {
                const int64_t j = j0 + cg * AS_CPT + c;
                const float cnj = cns[cg * AS_CPT + c];
#pragma unroll
                for (int r = 0; r < AS_RPT; r++) {
                    const int rr = rg * AS_RPT + r;
                    if (j < k && rr < nrows && fmaf(-2.f, acc[r][c], cnj) <= lim[r]) pend |= 1u << (r * AS_CPT + c);
                }
            }
            if (!__syncthreads_or(pend != 0)) continue;
            for (;;) {
                // queue what fits; the rest waits for the next round
                const int np = __popc(pend);
                int pos = np ? atomicAdd(&s_qn, np) : 0;
                uint32_t rest = 0;
                for (uint32_t m = pend; m; m &= m - 1) {
                    const int bt = __ffs((int)m) - 1;
                    if (pos < DQ_CAP)
                        qi[pos] = (uint16_t)((rg * AS_RPT + bt / AS_CPT) * AS_TC + cg * AS_CPT + bt % AS_CPT);
                    else
                        rest |= 1u << bt;
                    pos++;
                }
                pend = rest;
                __syncthreads();
                const int nq = min(s_qn, DQ_CAP);
                for (int e = t; e < nq; e += 256) {
                    const int ee = qi[e];
                    const int rr = ee / AS_TC;
                    const double D = ref_dist_strided(xs + rr, AS_TR, I.c64 + (j0 + ee % AS_TC) * d, d);
                    qd[e] = D;
                    atomicMin(&sbD[rr], (unsigned long long)__double_as_longlong(D));
                }
                __syncthreads();
                for (int e = t; e < nq; e += 256) {
                    const int ee = qi[e];
                    const int rr = ee / AS_TC;
                    if ((unsigned long long)__double_as_longlong(qd[e]) == sbD[rr])
                        atomicMin(&tJ[rr], (int)(j0 + ee % AS_TC));
                }
                __syncthreads();
                if (t < AS_TR) {
                    if (tJ[t] != 0x7FFFFFFF) {
                        // a new smallest D: its smallest index; the same D again: the smaller index
                        sbJ[t] = sbD[t] < prevD[t] ? tJ[t] : min(sbJ[t], tJ[t]);
                        tJ[t] = 0x7FFFFFFF;
                    }
                    prevD[t] = sbD[t];
                }
                if (t == 0) s_qn = 0;
                if (!__syncthreads_or(pend != 0)) break;
            }
        }
        if (t < nrows) I.labels[s_rows[t]] = sbJ[t] == 0x7FFFFFFF ? -1 : sbJ[t];
    }
}

__global__ void k_scatter_m(const int32_t *__restrict__ rows, const float *__restrict__ m,
                            const unsigned long long *__restrict__ n, float *__restrict__ mrow) {
    const int64_t nf = (int64_t)*n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += (int64_t)gridDim.x * blockDim.x)
        mrow[rows[q]] = m[q];
}

// ---- grouping a flag list by instance (device-side, graph friendly) --------
__global__ void k_flag_count(const int32_t *__restrict__ flags, const unsigned long long *__restrict__ n_flag,
                             const int64_t *__restrict__ row_off, int count, int *__restrict__ cnt) {
    const int64_t nf = (int64_t)*n_flag;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[find_inst(row_off, count, flags[q])], 1);
}

// one block: segment offsets and 128-row units per instance; cursor[i] =
// segment start for the scatter
__global__ void __launch_bounds__(1024) k_flag_units(const int *__restrict__ cnt, int count, int64_t *__restrict__ cursor,
                                                     int *__restrict__ unit_inst, int64_t *__restrict__ unit_start,
                                                     int *__restrict__ unit_cnt, int *__restrict__ n_units) {
    __shared__ int64_t seg_carry, unit_carry;
    __shared__ int64_t s_seg[1024], s_unit[1024];
    if (threadIdx.x == 0) seg_carry = unit_carry = 0;
    __syncthreads();
    for (int base = 0; base < count; base += 1024) {
        const int i = base + threadIdx.x;
        const int64_t c = i < count ? cnt[i] : 0;
        const int64_t nu = (c + AS_TR - 1) / AS_TR;
        s_seg[threadIdx.x] = c;
        s_unit[threadIdx.x] = nu;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive scans
            const int64_t a = threadIdx.x >= o ? s_seg[threadIdx.x - o] : 0;
            const int64_t b = threadIdx.x >= o ? s_unit[threadIdx.x - o] : 0;
            __syncthreads();
            s_seg[threadIdx.x] += a;
            s_unit[threadIdx.x] += b;
            __syncthreads();
        }
        const int64_t so = seg_carry + s_seg[threadIdx.x] - c, uo = unit_carry + s_unit[threadIdx.x] - nu;
        if (i < count) {
            cursor[i] = so;
            for (int64_t q = 0; q < nu; q++) {
                unit_inst[uo + q] = i;
                unit_start[uo + q] = so + q * AS_TR;
                unit_cnt[uo + q] = (int)min((int64_t)AS_TR, c - q * AS_TR);
            }
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            seg_carry += s_seg[1023];
            unit_carry += s_unit[1023];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_units = (int)unit_carry;
}

__global__ void k_flag_scatter(const int32_t *__restrict__ flags, const unsigned long long *__restrict__ n_flag,
                               const int64_t *__restrict__ row_off, int count, int64_t *__restrict__ cursor,
                               int32_t *__restrict__ grows) {
    const int64_t nf = (int64_t)*n_flag;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = flags[q];
        grows[atomicAdd((unsigned long long *)&cursor[find_inst(row_off, count, r)], 1ull)] = r;
    }
}

// Exact decision for flagged objects, one warp per object, one centre per
// lane (the row in shared memory): an FP32 pass over all centres finds the
// smallest fast value m; a second pass takes every centre whose fast value
// is within the FP32 window of m and decides among them with the FP64
// reference distance, ties to the smaller index.  Flag entries are global rows; instance i owns rows
// [row_off[i], row_off[i + 1]).  d <= 256.
// With flag_m, entry q brings the smallest fast value of its row from the
// tiled FP32 pass and the first pass is skipped.  Any fast value f' of any
// centre j' serves as m: the winner j* has fast(j*) <= D(j*) + W <= D(j') + W
// <= f' + 2W, W the rigorous FP32 window (both passes are within W of the
// exact distance whatever their summation order).  NaN: no finite value.
constexpr int RC_MAXD = 256;
__global__ void __launch_bounds__(256) k_assign_recheck(const RInst *__restrict__ R,
                                                        const int64_t *__restrict__ row_off, int count,
                                                        const int32_t *__restrict__ flag_rows,
                                                        const float *__restrict__ flag_m,
                                                        const unsigned long long *__restrict__ n_flag) {
    __shared__ __align__(16) float xs[8][RC_MAXD];  // the warp's row
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = (int64_t)*n_flag;
    for (int64_t q = warp; q < nf; q += nw) {
        const int64_t grow = flag_rows[q];
        const RInst &I = R[find_inst(row_off, count, grow)];
        const int64_t row = grow - I.row_base;
        const int d = I.d;
        const int64_t k = I.k;
        const float *xr = I.x + row * I.ldx;
        float xv[RC_MAXD / 32];
        float xs2 = 0.f;
#pragma unroll
        for (int u = 0; u < RC_MAXD / 32; u++) {
            const int t = lane + 32 * u;
            xv[u] = t < d ? xr[t] : 0.f;
            if (t < d) xs[wib][t] = xv[u];
            xs2 = fmaf(xv[u], xv[u], xs2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xs2 += __shfl_xor_sync(0xffffffffu, xs2, o);
        __syncwarp();
        const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
        const float cmax = __uint_as_float(*I.cmax_bits);
        // fast value of centre j, one centre per lane: the row is read from
        // shared memory (a broadcast), the centre from its own row
        const float *xw = xs[wib];
        const bool v4 = (d & 3) == 0 && (((uintptr_t)I.c32) & 15) == 0;
        auto fast = [&](int64_t j) {
            const float *cr = I.c32 + j * d;
            float dot = 0.f;
            if (v4) {
                for (int t = 0; t < d; t += 4) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(cr + t);
                    const float4 x4 = *reinterpret_cast<const float4 *>(xw + t);
                    dot = fmaf(x4.x, c4.x, dot);
                    dot = fmaf(x4.y, c4.y, dot);
                    dot = fmaf(x4.z, c4.z, dot);
                    dot = fmaf(x4.w, c4.w, dot);
                }
            } else {
                for (int t = 0; t < d; t++) dot = fmaf(xw[t], cr[t], dot);
            }
            return fmaf(-2.f, dot, I.cn[j]);
        };
        float m = flag_m ? flag_m[q] : __int_as_float(0x7fc00000);
        if (m != m) {
            m = FLT_MAX;
            for (int64_t j0 = 0; j0 < k; j0 += 32) {
                const int64_t j = j0 + lane;
                if (j < k) m = fminf(m, fast(j));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        const float lim = m + 2.f * window_fp32(xn, cmax, d) * (1.f + 1e-6f);
        double bD = DBL_MAX;
        int bj = 0x7FFFFFFF;
        for (int64_t j0 = 0; j0 < k; j0 += 32) {
            const int64_t j = j0 + lane;
            // candidates: fast value within the window of m; the FP64
            // reference decides among them, each lane its own
            if (j < k && fast(j) <= lim) {
                const double D = ref_dist(xw, I.c64 + j * d, d);
                if (D < bD || (D == bD && (int)j < bj)) {
                    bD = D;
                    bj = (int)j;
                }
            }
        }
        // warp argmin, ties to the smaller index
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double D2 = __shfl_xor_sync(0xffffffffu, bD, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
            if (D2 < bD || (D2 == bD && j2 < bj)) {
                bD = D2;
                bj = j2;
            }
        }
        // no candidate with a distance below +inf (non-finite input): -1,
        // as the reference argmin that never improves on +inf
        if (lane == 0) I.labels[row] = bj == 0x7FFFFFFF ? -1 : bj;
        __syncwarp();
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

// running sum sh + sl of non-negative FP32 values with each addition's
// rounding error kept (TwoSum): relative error about 2^-23 for any count,
// in FP32 operations only
__device__ __forceinline__ void csum_add(float &sh, float &sl, float v) {
    const float t = __fadd_rn(sh, v);
    const float bb = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(v, bb));
    sh = t;
    sl = __fadd_rn(sl, err);
}

// Lane partials of four rows' distances to their labelled centres (rows
// i[q] < n; d <= 128, rows and centre halves 16-byte aligned): lane l holds
// coordinates 4l .. 4l+3, diff = (x - c_hi) - c_lo, squares summed in FP32.
// Every row's label and coordinates are requested before any centre, so the
// four rows' loads are in flight together.
__device__ __forceinline__ void dist4_vec(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                          const float *__restrict__ chi, const float *__restrict__ clo, int64_t k,
                                          const int32_t *__restrict__ labels, const int64_t (&i)[4], float (&D)[4],
                                          bool (&ok)[4]) {
    const int lane = threadIdx.x & 31;
    const bool mine = 4 * lane < d;
    int j[4];
    float4 xv[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        j[q] = i[q] < n ? labels[i[q]] : -1;
        xv[q] = (i[q] < n && mine) ? *reinterpret_cast<const float4 *>(x + i[q] * ldx + 4 * lane)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        ok[q] = j[q] >= 0 && j[q] < k;  // uniform across the warp
        const bool use = ok[q] && mine;
        const float4 hv = use ? *reinterpret_cast<const float4 *>(chi + (int64_t)j[q] * d + 4 * lane)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 lv = use ? *reinterpret_cast<const float4 *>(clo + (int64_t)j[q] * d + 4 * lane)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        const float e0 = (xv[q].x - hv.x) - lv.x, e1 = (xv[q].y - hv.y) - lv.y;
        const float e2 = (xv[q].z - hv.z) - lv.z, e3 = (xv[q].w - hv.w) - lv.w;
        D[q] = use ? fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, fmaf(e0, e0, 0.f)))) : 0.f;
    }
}

// per-object distance to its centre, warp per object, lanes over
// coordinates: diff = (x - c_hi) - c_lo, squares accumulated in FP32; the
// warp's distances in a compensated FP32 sum, block partial sums (FP64) and
// maxima, reduced on one block in a fixed order
__global__ void __launch_bounds__(256) k_assign_stats(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                                      const float *__restrict__ chi, const float *__restrict__ clo,
                                                      int64_t k, const int32_t *__restrict__ labels,
                                                      double *__restrict__ part_sum, float *__restrict__ part_max) {
    __shared__ double ss[8];
    __shared__ float sm_[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float sh = 0.f, sl = 0.f;  // compensated FP32 sum of the warp's distances
    float mx = 0.f;
    // rows, centre halves and the row pitch 16-byte aligned: a lane takes 4
    // consecutive coordinates per load (same summation depth per row)
    const bool vec = ((d & 3) == 0) && ((ldx & 3) == 0) && (((uintptr_t)x & 15) == 0) &&
                     (((uintptr_t)chi & 15) == 0) && (((uintptr_t)clo & 15) == 0);
    // four rows in flight per warp (independent loads and reductions)
    for (int64_t i0 = warp; i0 < n; i0 += 4 * nw) {
        float D[4];
        bool ok[4];
        if (vec && d <= 128) {
            const int64_t iq[4] = {i0, i0 + nw, i0 + 2 * nw, i0 + 3 * nw};
            dist4_vec(x, ldx, n, d, chi, clo, k, labels, iq, D, ok);
        } else {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int64_t i = i0 + q * nw;
            const int j = i < n ? labels[i] : -1;
            ok[q] = j >= 0 && j < k;  // uniform across the warp
            D[q] = 0.f;
            if (ok[q]) {
                const float *xr = x + i * ldx;
                const float *h = chi + (int64_t)j * d;
                const float *l = clo + (int64_t)j * d;
                if (vec) {
                    for (int t = 4 * lane; t < d; t += 128) {
                        const float4 xv = *reinterpret_cast<const float4 *>(xr + t);
                        const float4 hv = *reinterpret_cast<const float4 *>(h + t);
                        const float4 lv = *reinterpret_cast<const float4 *>(l + t);
                        const float e0 = (xv.x - hv.x) - lv.x, e1 = (xv.y - hv.y) - lv.y;
                        const float e2 = (xv.z - hv.z) - lv.z, e3 = (xv.w - hv.w) - lv.w;
                        D[q] = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, fmaf(e0, e0, D[q]))));
                    }
                } else {
                    for (int t = lane; t < d; t += 32) {
                        const float e = (xr[t] - h[t]) - l[t];
                        D[q] = fmaf(e, e, D[q]);
                    }
                }
            }
        }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; q++) D[q] += __shfl_xor_sync(0xffffffffu, D[q], o);
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (ok[q]) {
                csum_add(sh, sl, D[q]);
                mx = fmaxf(mx, D[q]);
            }
    }
    if (lane == 0) {
        ss[wib] = (double)sh + (double)sl;
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
__global__ void __launch_bounds__(256, 4) k_assign_stats_batch(const SInst *__restrict__ S, const int2 *__restrict__ units,
                                                            int64_t nunits, double *__restrict__ part_sum,
                                                            float *__restrict__ part_max) {
    __shared__ double ss[8];
    __shared__ float sm_[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int2 un = units[u];
        const SInst &I = S[un.x];
        float sh = 0.f, sl = 0.f;  // compensated FP32 sum of the warp's distances
        float mx = 0.f;
        const bool vec = I.d <= 128 && ((I.d & 3) == 0) && ((I.ldx & 3) == 0) && (((uintptr_t)I.x & 15) == 0) &&
                         (((uintptr_t)I.chi & 15) == 0) && (((uintptr_t)I.clo & 15) == 0);
        // rows wib, wib + 8, ... of the unit, four in flight per warp
        for (int r0 = wib; r0 < 128; r0 += 32) {
            float D[4];
            bool ok[4];
            if (vec) {
                const int64_t b = (int64_t)un.y * 128 + r0;
                const int64_t iq[4] = {b, b + 8, b + 16, b + 24};
                dist4_vec(I.x, I.ldx, I.n, I.d, I.chi, I.clo, I.k, I.labels, iq, D, ok);
            } else {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int64_t i = (int64_t)un.y * 128 + r0 + 8 * q;
                const int j = i < I.n ? I.labels[i] : -1;
                ok[q] = j >= 0 && j < I.k;  // uniform across the warp
                D[q] = 0.f;
                if (ok[q]) {
                    const float *xr = I.x + i * I.ldx;
                    const float *h = I.chi + (int64_t)j * I.d;
                    const float *l = I.clo + (int64_t)j * I.d;
                    for (int t = lane; t < I.d; t += 32) {
                        const float e = (xr[t] - h[t]) - l[t];
                        D[q] = fmaf(e, e, D[q]);
                    }
                }
            }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int q = 0; q < 4; q++) D[q] += __shfl_xor_sync(0xffffffffu, D[q], o);
            }
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (ok[q]) {
                    csum_add(sh, sl, D[q]);
                    mx = fmaxf(mx, D[q]);
                }
        }
        __syncthreads();
        if (lane == 0) {
            ss[wib] = (double)sh + (double)sl;
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

// Per-cluster radius (Sect. 4.1): for every object its distance to its
// centre as in k_assign_stats (warp per object, diff = (x - c_hi) - c_lo,
// squares in FP32), and per label the largest one by an atomic maximum on the
// bits of the non-negative float.
__global__ void __launch_bounds__(256) k_cluster_rmax(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                                      const float *__restrict__ chi, const float *__restrict__ clo,
                                                      int64_t k, const int32_t *__restrict__ labels,
                                                      unsigned *__restrict__ rmax) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nw) {
        const int j = labels[i];
        if (j < 0 || j >= k) continue;  // warp-uniform
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
        if (lane == 0) atomicMax(&rmax[j], __float_as_uint(D));
    }
}

__global__ void k_cluster_sqrt(int64_t k, const unsigned *__restrict__ rmax, double *__restrict__ radius) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x)
        radius[j] = sqrt((double)__uint_as_float(rmax[j]));
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

// ---- extra passes of assignment (Sect. 5) --------------------------------
// members grouped by label: key = label (k for -1), id; counts per label
__global__ void k_label_keys(int64_t n, const int32_t *__restrict__ labels, int64_t k, uint64_t *__restrict__ key,
                             uint32_t *__restrict__ ids, unsigned long long *__restrict__ cnt, int *__restrict__ bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = labels[i];
        if (l < -1 || l >= k) {
            atomicExch(bad, 1);
            l = -1;
        }
        key[i] = l < 0 ? (uint64_t)k : (uint64_t)l;
        ids[i] = (uint32_t)i;
        if (l >= 0) atomicAdd(&cnt[l], 1ull);
    }
}

// sort key of centre j: descending member count, then ascending index
__global__ void k_size_order(int64_t k, const unsigned long long *__restrict__ cnt, uint64_t *__restrict__ key) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t cj = cnt[j] > 0xFFFFFFFFull ? 0xFFFFFFFFull : cnt[j];
        key[j] = ((0xFFFFFFFFull - cj) << 32) | (uint64_t)j;
    }
}

// centre j <- mean of its members (ascending id, the seeds' centroid sum);
// no member: unchanged.  Work item = (centre, slice of 32 coordinates), one
// warp per item, lane = coordinate; each lane's sum is the sequential FP64
// chain s <- RN(s + x_i) over the centre's members in ascending id.
//
// An FP64 add on this part takes 60-170 cycles in a dependent chain (longer
// for operands of mixed exponents), which would bound the pass by the
// largest cluster's member count times that latency.  So each 32-member
// chunk first runs the chain in 64-bit integers, in a unit 2^g that divides
// s and every x_i of the chunk (the finer of s's lowest set bit and the
// finest ulp among the x_i): s = T 2^g.  While every partial sum T + R_1 +
// ... + R_i (R_i = x_i / 2^g) stays below 2^53 in magnitude, each partial
// sum is exactly representable in FP64, so each RN step is exact and the
// chain equals the integer sum (binade and sign changes included).  The
// first step that breaks this (a sum reaching 2^53 units, where rounding may
// start; an x_i too far above the unit or not finite), and every step after
// it in the chunk, runs as the FP64 add itself; so the result is the FP64
// chain bit for bit.  The integer sum is accumulated unconditionally (a
// 64-bit add is the only loop-carried step) and the failures collected in a
// bit mask.
//
// Each work item is served by a pair of warps: a producer (fetches the item,
// loads the member ids four stages ahead, copies 32 member rows per stage
// into the pair's ring of UC_S stages with 16-byte cp.async, 4 rows per
// instruction) and a consumer (the chain above, a stage at a time), so the
// consumer's single instruction stream carries only the sums.  Stage hand-off
// by mbarriers: "full" completes when the producer's 32 lanes' copies have
// landed (cp.async.mbarrier.arrive.noinc) and its header is written, "empty"
// when the consumer is done with the stage; every wait is bounded (on expiry
// the kernel records GEEK_ERR_TIMEOUT and both warps stop).  The first wave of
// items goes to pairs pair-in-block major, so the slices of one centre start
// on different SMs; later items come from an atomic counter, largest centre
// first (order: centre indices by descending member count).
constexpr int UC_P = 4, UC_T = 64 * UC_P, UC_B = 32, UC_S = 8;
constexpr int UC_STAGE = UC_B * 32;                                    // floats per stage
constexpr int UC_SMEM = UC_P * UC_S * UC_STAGE * (int)sizeof(float);   // 128 KB of rings

// a stage's header: which item and which 32 members
struct UcHdr {
    int64_t j, cj;  // centre, its member count (cj < 0: no more items)
    int32_t t0, g;  // first coordinate of the slice, member group
};

// x / 2^g as a signed integer, x = +-mx 2^u with base = 150 + g and u >= g:
// exact for u - g <= 38 (then |x / 2^g| < 2^62); bad beyond that or when x
// is not finite
__device__ __forceinline__ int64_t units_of(float x, int base, bool &bad) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    const uint32_t mx = (b & 0x7FFFFFu) | ((uint32_t)min(e, 1) << 23);
    const int lsh = max(e, 1) - base;  // u - g >= 0
    bad = lsh > 38 || e == 0xFF;
    const int64_t R = (int64_t)((uint64_t)mx << (lsh & 63));
    return (b >> 31) ? -R : R;
}

// s <- RN(...RN(RN(s + v[0]) + v[1]) ... + v[ma - 1]) in FP64, ma <= 32 (a
// lane with act = false, past the last coordinate, takes no FP64 step and
// so holds up no other lane)
// FULL: ma == UC_B, every step unpredicated and the one-check sum a tree.
template <bool FULL>
__device__ __forceinline__ double chain_chunk(double s, const float (&v)[UC_B], int ma, bool act) {
    if (FULL) ma = UC_B;
    constexpr uint64_t M52 = (1ull << 52) - 1;
    const uint64_t bits = (uint64_t)__double_as_longlong(s);
    const int E = (int)((bits >> 52) & 0x7FF);
    const bool zero = bits == 0;  // +0 (the running sum never becomes -0)
    // integer steps from +0 or from a normal s well inside the range
    bool fast = zero || (E > 64 && E < 0x7FE - 64);
    const uint64_t M = (bits & M52) | (1ull << 52);
    // the unit 2^g: the finest ulp among the chunk's values and s's lowest set bit
    // (tree reductions: no 32-long dependency chain)
    int ua[UC_B], ea[UC_B];
#pragma unroll
    for (int m = 0; m < UC_B; m++) {
        const int e = (int)((__float_as_uint(v[m]) >> 23) & 0xFFu);
        ua[m] = m < ma ? max(e, 1) : 0x7FFFFFFF;
        ea[m] = m < ma ? e : 0;
    }
#pragma unroll
    for (int w = 1; w < UC_B; w <<= 1)
#pragma unroll
        for (int m = 0; m < UC_B; m += 2 * w) {
            ua[m] = min(ua[m], ua[m + w]);
            ea[m] = max(ea[m], ea[m + w]);
        }
    const int umin = ua[0], emax = ea[0];
    const int qs = E - 1075;
    const int g = zero ? umin - 150 : min(umin - 150, qs + __ffsll((long long)M) - 1);
    int64_t T0 = 0;
    if (!zero) {
        const int sh = qs - g;  // > 0: s's ulp is coarser than a value's (s then needs more than 53 bits)
        fast = fast && sh <= 10;
        const uint64_t a0 = sh >= 0 ? (M << min(sh, 10)) : (M >> min(-sh, 63));  // exact: g <= s's lowest set bit
        T0 = (bits >> 63) ? -(int64_t)a0 : (int64_t)a0;
    }
    const int base = 150 + g;
    // every |x_i / 2^g| < 2^(24 + lmax) (0 <= lmax): if |T0| + 32 2^(24 + lmax)
    // < 2^53, no partial sum can reach 2^53 and the chunk is one exact
    // integer sum (any order); otherwise each partial sum is checked
    const int lmax = max(emax, 1) - base;
    const uint64_t aT0 = (uint64_t)(T0 < 0 ? -T0 : T0);
    const bool easy = fast && emax != 0xFF && lmax <= 23 && aT0 + (1ull << (29 + lmax)) < (1ull << 53);
    int64_t T = T0;
    int f = ma;  // first step that takes the FP64 add
    if (easy && FULL) {
        int64_t r[UC_B];
#pragma unroll
        for (int m = 0; m < UC_B; m++) {
            bool bad;
            r[m] = units_of(v[m], base, bad);
        }
#pragma unroll
        for (int w = 1; w < UC_B; w <<= 1)
#pragma unroll
            for (int m = 0; m < UC_B; m += 2 * w) r[m] += r[m + w];
        T += r[0];
    } else if (easy) {
        int64_t p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
        for (int m = 0; m < UC_B; m += 4) {
            bool bad;
            if (m < ma) T += units_of(v[m], base, bad);
            if (m + 1 < ma) p1 += units_of(v[m + 1], base, bad);
            if (m + 2 < ma) p2 += units_of(v[m + 2], base, bad);
            if (m + 3 < ma) p3 += units_of(v[m + 3], base, bad);
        }
        T += p1 + p2 + p3;
    } else if (act) {
        uint32_t fail = fast ? 0u : 1u;
#pragma unroll
        for (int m = 0; m < UC_B; m++) {
            if (m < ma) {
                bool bad;
                T += units_of(v[m], base, bad);
                // |T| < 2^53: every partial sum is an FP64 value, each RN step exact
                const bool ok = !bad && (uint64_t)(T + (int64_t)((1ull << 53) - 1)) < (1ull << 54) - 1;
                if (!ok) fail |= 1u << m;
            }
        }
        f = fail ? __ffs((int)fail) - 1 : ma;
    }
    if (f < ma && f > 0) {  // the integer sum up to step f - 1
        T = T0;
#pragma unroll
        for (int m = 0; m < UC_B; m++)
            if (m < f) {
                bool bad;
                T += units_of(v[m], base, bad);
            }
    }
    double t = s;
    if (f > 0 && act) {  // T 2^g, |T| < 2^53, as an FP64 value (exact)
        const uint64_t a = (uint64_t)(T < 0 ? -T : T);
        if (a == 0) {
            t = 0.0;  // an exactly cancelling sum is +0 under RN
        } else {
            const int p = 64 - __clzll((long long)a);  // <= 53
            const uint64_t mant = (a << (53 - p)) & M52;
            t = __longlong_as_double(
                (long long)(((uint64_t)(T < 0) << 63) | ((uint64_t)(g + 1075 + p - 53) << 52) | mant));
        }
    }
    if (__all_sync(0xffffffffu, f >= ma)) return t;
    const int fw = __reduce_min_sync(0xffffffffu, f);  // warp-uniform bound of the FP64 tail
#pragma unroll
    for (int m = 0; m < UC_B; m++)
        if (m >= fw && m < ma && m >= f) t = __dadd_rn(t, widen_f32(v[m]));
    return t;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void cp_async_bar_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

__global__ void __launch_bounds__(UC_T) k_update_centres(const float *__restrict__ x, int64_t ldx, int d, int64_t k,
                                                         const int64_t *__restrict__ off,
                                                         const unsigned long long *__restrict__ cnt,
                                                         const int32_t *__restrict__ ids, const uint64_t *__restrict__ order,
                                                         unsigned long long *__restrict__ next, double *__restrict__ c,
                                                         int *__restrict__ err) {
    extern __shared__ float uc_ring[];  // [UC_P][UC_S][32 rows][32 floats]
    __shared__ UcHdr hdr[UC_P][UC_S];
    __shared__ uint64_t full[UC_P][UC_S], empty[UC_P][UC_S];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool producer = warp >= UC_P;
    const int pr = producer ? warp - UC_P : warp;  // the pair
    float *ring = uc_ring + (size_t)pr * UC_S * UC_STAGE;
    if (threadIdx.x < UC_P * UC_S) {
        mbar_init(&full[threadIdx.x / UC_S][threadIdx.x % UC_S], 33);  // 32 copy arrivals + the header
        mbar_init(&empty[threadIdx.x / UC_S][threadIdx.x % UC_S], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const int nsl = (d + 31) >> 5;
    const int64_t nitems = k * nsl;
    if (producer) {
        const uint32_t ring_s = su32(ring);
        const bool vec = (((uintptr_t)x & 15) == 0) && ((ldx & 3) == 0);
        const int64_t np = (int64_t)gridDim.x * UC_P;
        int64_t it = (int64_t)pr * gridDim.x + blockIdx.x;  // first wave: slices of a centre on different SMs
        uint32_t sn = 0;                                    // stages issued by this pair
        bool ok = true;
        for (;;) {
            const bool done = it >= nitems;
            int64_t j = 0, cj = 0;
            int t0 = 0;
            if (!done) {
                j = (int64_t)(order[it / nsl] & 0xFFFFFFFFull);
                t0 = (int)(it % nsl) * 32;
                cj = (int64_t)cnt[j];
            }
            const int width = min(32, d - t0);
            const int col = (lane & 7) * 4;  // this lane's 16 bytes of a row slice (vector copies)
            const int nbytes = max(0, min(16, (width - col) * 4));
            const int32_t *mid = ids + (done ? 0 : off[j]);
            const float *xs = x + t0;
            const int64_t ng = done ? 1 : (cj + UC_B - 1) / UC_B;  // the end marker takes one stage
            auto ld_id = [&](int64_t g) -> int32_t {
                const int64_t q = g * UC_B + lane;
                return (!done && q < cj) ? mid[q] : 0;
            };
            int32_t id0 = ld_id(0), id1 = ld_id(1), id2 = ld_id(2), id3 = ld_id(3);
            for (int64_t g = 0; g < ng && ok; g++, sn++) {
                const int st = (int)(sn % UC_S);
                const uint32_t use = sn / UC_S;
                if (lane == 0) ok = mbar_wait(&empty[pr][st], (use & 1) ^ 1, err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                const int32_t my = id0;
                id0 = id1;
                id1 = id2;
                id2 = id3;
                id3 = ld_id(g + 4);
                if (!done) {
                    const int rows = (int)min((int64_t)UC_B, cj - g * UC_B);
                    const uint32_t sb = ring_s + (uint32_t)(st * UC_STAGE * sizeof(float));
                    if (vec) {
#pragma unroll
                        for (int i = 0; i < UC_B / 4; i++) {
                            const int rr = 4 * i + (lane >> 3);
                            const int32_t r = __shfl_sync(0xffffffffu, my, rr);
                            if (rr < rows)
                                cp_async16(sb + (uint32_t)(rr * 32 + col) * 4u, xs + (int64_t)r * ldx + (nbytes ? col : 0),
                                           nbytes);
                        }
                    } else {
#pragma unroll 8
                        for (int rr = 0; rr < UC_B; rr++) {
                            const int32_t r = __shfl_sync(0xffffffffu, my, rr);
                            if (rr < rows)
                                cp_async4(sb + (uint32_t)(rr * 32 + lane) * 4u, xs + (int64_t)r * ldx + (lane < width ? lane : 0),
                                          lane < width ? 4 : 0);
                        }
                    }
                }
                cp_async_bar_arrive(&full[pr][st]);  // when this lane's copies have landed
                if (lane == 0) {
                    hdr[pr][st] = UcHdr{j, done ? -1 : cj, t0, (int32_t)g};
                    mbar_arrive(&full[pr][st]);
                }
            }
            if (done || !ok) break;
            unsigned long long got = 0;
            if (lane == 0) got = atomicAdd(next, 1ull);
            it = np + (int64_t)__shfl_sync(0xffffffffu, got, 0);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // own copies landed before the block ends
    } else {
        double s = 0.0;
        for (uint32_t sn = 0;; sn++) {
            const int st = (int)(sn % UC_S);
            const uint32_t use = sn / UC_S;
            // lane 0 waits; __syncwarp then orders the other lanes' reads after
            // its acquire of the phase (the copies were the producer's)
            int okw = 0;
            if (lane == 0) okw = mbar_wait(&full[pr][st], use & 1, err);
            okw = __shfl_sync(0xffffffffu, okw, 0);
            __syncwarp();
            if (!okw) break;
            const UcHdr h = hdr[pr][st];
            if (h.cj < 0) break;
            const int width = min(32, d - h.t0);
            if (h.g == 0) s = 0.0;
            const float *src = ring + st * UC_STAGE + lane;
            float v[UC_B];
#pragma unroll
            for (int m = 0; m < UC_B; m++) v[m] = src[m * 32];
            const int ma = (int)min((int64_t)UC_B, h.cj - (int64_t)h.g * UC_B);
            s = ma == UC_B ? chain_chunk<true>(s, v, ma, lane < width) : chain_chunk<false>(s, v, ma, lane < width);
            __syncwarp();  // every lane's reads done before the stage is refilled
            if (lane == 0) mbar_arrive(&empty[pr][st]);
            if ((int64_t)(h.g + 1) * UC_B >= h.cj && lane < width) c[h.j * d + h.t0 + lane] = __ddiv_rn(s, (double)h.cj);
        }
    }
}

geek_status refine_dense(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d, double *centres,
                         int64_t k, int passes, int precision, int32_t *labels, geek_assign_stats *stats,
                         cudaStream_t st) {
    for (int pass = 0; pass < passes && n > 0 && k > 0; pass++) {
        Scratch ps(ctx, st);
        uint64_t *key;
        uint32_t *ids;
        unsigned long long *cnt;
        int64_t *off;
        int *bad;
        GK_TRY(ps.alloc(&key, n));
        GK_TRY(ps.alloc(&ids, n));
        GK_TRY(ps.alloc(&cnt, k));
        GK_TRY(ps.alloc(&off, k));
        GK_TRY(ps.alloc(&bad, 1));
        EvTimer tg(ctx, "refine.group", st);
        GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * k, st));
        GK_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), st));
        GK_COUNT();
        k_label_keys<<<grid_for(n, 256, ctx->num_sms), 256, 0, st>>>(n, labels, k, key, ids, cnt, bad);
        GK_LAUNCH(ctx);
        GK_TRY(radix_sort_segments(ctx, ps, 1, n, &key, nullptr, &ids, bit_length_u64((uint64_t)k), st));
        GK_TRY(exclusive_scan_i64(ctx, ps, (const int64_t *)cnt, off, k, nullptr, st));
        uint64_t *order;
        GK_TRY(ps.alloc(&order, k));
        GK_COUNT();
        k_size_order<<<grid_for(k, 256, ctx->num_sms), 256, 0, st>>>(k, cnt, order);
        GK_LAUNCH(ctx);
        GK_TRY(radix_sort_segments(ctx, ps, 1, k, &order, nullptr, nullptr, 64, st));
        tg.stop();
        unsigned long long *next;
        int *uc_err;
        GK_TRY(ps.alloc(&next, 1));
        GK_TRY(ps.alloc(&uc_err, 1));
        GK_CUDA(ctx, cudaMemsetAsync(next, 0, sizeof(unsigned long long), st));
        GK_CUDA(ctx, cudaMemsetAsync(uc_err, 0, sizeof(int), st));
        static bool uc_attr = false;
        if (!uc_attr) {
            GK_CUDA(ctx, cudaFuncSetAttribute(k_update_centres, cudaFuncAttributeMaxDynamicSharedMemorySize, UC_SMEM));
            uc_attr = true;
        }
        EvTimer tu(ctx, "kernel.update_centres", st);
        GK_COUNT();
        k_update_centres<<<(unsigned)std::min<int64_t>((k * ((d + 31) / 32) + UC_P - 1) / UC_P, (int64_t)ctx->num_sms),
                           UC_T, UC_SMEM, st>>>(x, ldx, d, k, off, cnt, (const int32_t *)ids, order, next, centres,
                                                uc_err);
        GK_LAUNCH(ctx);
        tu.stop();
        int h_bad = 0, h_uc = 0;
        GK_CUDA(ctx, cudaMemcpyAsync(&h_bad, bad, sizeof h_bad, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaMemcpyAsync(&h_uc, uc_err, sizeof h_uc, cudaMemcpyDeviceToHost, st));
        GK_TRY(sort_err_check(ctx, st));  // synchronises st
        if (h_bad) return set_error(ctx, GEEK_ERR_INVALID, "a label outside [-1, k)");
        if (h_uc) return set_error(ctx, (geek_status)h_uc, "centre update: a pipeline wait timed out");
        EvTimer ta(ctx, "refine.assign", st);
        // the statistics describe the last pass only
        GK_TRY(assign_dense_centres(ctx, ps, x, ldx, n, d, centres, k, precision, labels,
                                    pass + 1 == passes ? stats : nullptr, st));
    }
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
    if (precision != GEEK_PREC_FP32 && precision != GEEK_PREC_BF16 && precision != GEEK_PREC_BF16X3)
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
    float *flag_m = nullptr;  // the FP32 pass's smallest value per flagged row
    unsigned long long *n_flag;
    GK_TRY(scr.alloc(&flag_rows, n));
    if (precision == GEEK_PREC_FP32) GK_TRY(scr.alloc(&flag_m, n));
    GK_TRY(scr.alloc(&n_flag, 1));
    GK_CUDA(ctx, cudaMemsetAsync(n_flag, 0, sizeof(unsigned long long), st));
    if (precision == GEEK_PREC_BF16 || precision == GEEK_PREC_BF16X3) {
        GK_TRY(assign_tc_bf16(ctx, scr, x, ldx, n, d, centres, k, precision == GEEK_PREC_BF16X3, labels, flag_rows,
                              n_flag, st));
    } else {
        const size_t smem = (size_t)d * AS_TR * sizeof(float) + (size_t)AS_KC * AS_TC * sizeof(float);
        GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EvTimer tk(ctx, "kernel.assign_fp32", st);
        tk.work = 2.0 * (double)n * (double)k * (double)d;
        FArgs A{x, ldx, n, d, c32, cn, k, cmax, labels, flag_rows, flag_m, n_flag, ceil_div(n, AS_TR)};
        GK_COUNT();
        k_assign_fp32<false><<<(unsigned)A.ntiles, 256, smem, st>>>(A, GatherUnits{});
        GK_LAUNCH(ctx);
    }
    unsigned long long h_flag = 0, h_fp64 = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_flag, n_flag, sizeof h_flag, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    DecideBufs db;
    if (h_flag) {
        GK_TRY(decide_bufs_alloc(ctx, &scr, 1, n, db));
        if (precision == GEEK_PREC_FP32) {
            // the FP32 pass already applied the FP32 window: straight to FP64
            const int blocks = (int)std::min<unsigned long long>(ceil_div((int64_t)h_flag, 8), (unsigned long long)ctx->num_sms * 8);
            EvTimer tk(ctx, "kernel.assign_recheck", st);
            GK_COUNT();
            k_assign_recheck<<<blocks, 256, 0, st>>>(ri, roff, 1, flag_rows, flag_m, n_flag);
            GK_LAUNCH(ctx);
            h_fp64 = h_flag;
        } else {
            GK_TRY(decide_flags(ctx, ri, roff, 1, d, flag_rows, n_flag, db, st));
        }
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
        if (h_flag && precision != GEEK_PREC_FP32)
            GK_CUDA(ctx, cudaMemcpyAsync(&h_fp64, db.n_flag2, sizeof h_fp64, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        stats->sse = h[0];
        stats->radius_max = h[1];
        stats->k = k;
        stats->n_recheck_rows = (int64_t)h_flag;
        stats->n_fp64_rows = (int64_t)h_fp64;
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

geek_status decide_bufs_alloc(geek_ctx *ctx, Scratch *scr, int count, int64_t n_total, DecideBufs &B) {
    const int64_t nu = ceil_div(n_total, AS_TR) + count;
    auto al = [&](auto **p, size_t c) -> geek_status {
        if (scr) return scr->alloc(p, c);
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(c * sizeof(**p), 16)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, GEEK_ERR_NOMEM, "decision buffers");
        }
        B.owned.push_back(q);
        *p = (std::remove_reference_t<decltype(*p)>)q;
        return GEEK_OK;
    };
    GK_TRY(al(&B.cnt, count));
    GK_TRY(al(&B.cursor, count));
    GK_TRY(al(&B.unit_inst, nu));
    GK_TRY(al(&B.unit_start, nu));
    GK_TRY(al(&B.unit_cnt, nu));
    GK_TRY(al(&B.n_units, 1));
    GK_TRY(al(&B.grows, std::max<int64_t>(n_total, 1)));
    GK_TRY(al(&B.flags2, std::max<int64_t>(n_total, 1)));
    GK_TRY(al(&B.flags2_m, std::max<int64_t>(n_total, 1)));
    GK_TRY(al(&B.mrow, std::max<int64_t>(n_total, 1)));
    GK_TRY(al(&B.n_flag2, 1));
    return GEEK_OK;
}

void decide_bufs_free(DecideBufs &B) {
    for (void *p : B.owned) cudaFree(p);
    B.owned.clear();
}

// Decides the flagged rows of a fast pass exactly: rows grouped by
// instance, a tiled FP32 pass (narrow FP32 window) over each group, then the
// FP64 reference for the rows still uncertain.  No host synchronisation.
geek_status decide_flags(geek_ctx *ctx, const RInst *R, const int64_t *row_off, int count, int dmax,
                         const int32_t *flags, const unsigned long long *n_flag, const DecideBufs &B,
                         cudaStream_t st) {
    EvTimer tk(ctx, "kernel.assign_recheck", st);
    const int g = ctx->num_sms * 4;
    GK_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(int) * count, st));
    GK_CUDA(ctx, cudaMemsetAsync(B.n_flag2, 0, sizeof(unsigned long long), st));
    GK_COUNT();
    k_flag_count<<<g, 256, 0, st>>>(flags, n_flag, row_off, count, B.cnt);
    GK_COUNT();
    k_flag_units<<<1, 1024, 0, st>>>(B.cnt, count, B.cursor, B.unit_inst, B.unit_start, B.unit_cnt, B.n_units);
    GK_COUNT();
    k_flag_scatter<<<g, 256, 0, st>>>(flags, n_flag, row_off, count, B.cursor, B.grows);
    GK_LAUNCH(ctx);
    const size_t smem = (size_t)dmax * AS_TR * sizeof(float) + (size_t)AS_KC * AS_TC * sizeof(float);
    static bool attr = false;
    if (!attr) {
        const size_t mx = (size_t)AS_MAXD * AS_TR * sizeof(float) + (size_t)AS_KC * AS_TC * sizeof(float);
        GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
        attr = true;
    }
    FArgs A{};
    A.flag_rows = B.flags2;
    A.flag_m = B.flags2_m;
    A.n_flag = B.n_flag2;
    GatherUnits U{R, B.grows, B.unit_inst, B.unit_start, B.unit_cnt, B.n_units};
    EvTimer t32(ctx, "kernel.assign_refine32", st);
    GK_COUNT();
    k_assign_fp32<true><<<ctx->num_sms * 2, 256, smem, st>>>(A, U);
    GK_LAUNCH(ctx);
    t32.stop();
    // the rows still uncertain, grouped by instance again, go to the tiled
    // FP64 decision with their smallest FP32 value
    static bool attr64 = false;
    if (!attr64) {
        const size_t mx =
            (size_t)AS_MAXD * AS_TR * sizeof(float) + (size_t)AS_KC * AS_TC * sizeof(float) + DQ_BYTES;
        GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_decide64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
        attr64 = true;
    }
    GK_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(int) * count, st));
    GK_COUNT();
    k_scatter_m<<<g, 256, 0, st>>>(B.flags2, B.flags2_m, B.n_flag2, B.mrow);
    GK_COUNT();
    k_flag_count<<<g, 256, 0, st>>>(B.flags2, B.n_flag2, row_off, count, B.cnt);
    GK_COUNT();
    k_flag_units<<<1, 1024, 0, st>>>(B.cnt, count, B.cursor, B.unit_inst, B.unit_start, B.unit_cnt, B.n_units);
    GK_COUNT();
    k_flag_scatter<<<g, 256, 0, st>>>(B.flags2, B.n_flag2, row_off, count, B.cursor, B.grows);
    EvTimer t64(ctx, "kernel.assign_decide64", st);
    GK_COUNT();
    k_assign_decide64<<<ctx->num_sms * 2, 256, smem + DQ_BYTES, st>>>(U, B.mrow);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

// radius[j] = sqrt(max over objects labelled j of their distance to centre
// j), 0 for a centre nobody is nearest to; labels outside [0, k) are skipped.
geek_status cluster_radius(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                           const double *centres, int64_t k, const int32_t *labels, double *radius, cudaStream_t st) {
    if (k == 0) return GEEK_OK;
    float *chi, *clo;
    unsigned *rmax;
    GK_TRY(scr.alloc(&chi, (size_t)k * d));
    GK_TRY(scr.alloc(&clo, (size_t)k * d));
    GK_TRY(scr.alloc(&rmax, k));
    GK_CUDA(ctx, cudaMemsetAsync(rmax, 0, sizeof(unsigned) * k, st));
    GK_COUNT();
    k_centre_split<<<grid_for(k * d, 256, ctx->num_sms), 256, 0, st>>>(centres, k * d, chi, clo);
    if (n > 0) {
        GK_COUNT();
        k_cluster_rmax<<<grid_for(n * 32, 256, ctx->num_sms), 256, 0, st>>>(x, ldx, n, d, chi, clo, k, labels, rmax);
    }
    GK_COUNT();
    k_cluster_sqrt<<<grid_for(k, 256, ctx->num_sms), 256, 0, st>>>(k, rmax, radius);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}
