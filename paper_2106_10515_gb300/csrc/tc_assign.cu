// Dense one-pass assignment on the 5th-generation tensor cores (tcgen05).
//
// S = X C^T in BF16 with FP32 accumulation in tensor memory, fused with a
// running arg-min epilogue over centre tiles; the FP64 decision of the
// exact argmin (Eq. 1) is left to objects whose best and second-best
// approximate values are closer than the rigorous error window.
//
// Persistent kernel, one CTA per SM, 10 warps:
//   warp 0     TMA producer: X row tiles (double buffered) and centre tiles
//              (2-stage ring), 128-byte swizzled, K-major, plus |c|^2 of
//              each centre tile by bulk copy
//   warp 1     MMA issuer: tcgen05.mma.cta_group::1.kind::f16, M=128, N=256,
//              into one of two TMEM accumulators (2 x 256 columns)
//   warps 2-9  epilogue: tcgen05.ld of the accumulator, d' = |c|^2 - 2 s,
//              per-row best / second-best over the centres; each warp reads
//              its TMEM lane quarter (warp % 4) and one half of the columns
//              (each column group is an independent running minimum per
//              row, so fewer groups mean fewer new-best rescans)
// Every mbarrier wait is bounded: on expiry the kernel records
// GEEK_ERR_TIMEOUT, stops issuing work, drains its own copies and MMAs, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>

#include "internal.cuh"
#include "tc_ptx.cuh"

// One instance of the (batched) assignment.  Device copies are read by the
// kernel; CUtensorMap's 64-byte alignment keeps every array element aligned.
struct TcInst {
    CUtensorMap tmA;             // Xb: {Kp, n} bf16, box {64, 128}
    CUtensorMap tmB;             // Cb = -2 c: {Kp, kpad} bf16, box {64, N}
    CUtensorMap tmX;             // |c|^2 columns: {16, kpad} bf16, box {16, N}, 32-byte swizzle
    const float *xnorm;          // n: upper bound of |x|
    const unsigned *cmax_bits;   // max over real centres of |c|^2 (FP32 bits)
    int32_t *labels;             // n
    int64_t n, k;
    int64_t row_base;            // global row of local row 0 (flag list entries)
    int ntiles_c, Kp, d, N;      // centre tiles of N columns, padded d, d, tile N
};

// Per-instance conversion arguments (device copies).
struct TcXPrep {
    const float *x;
    int64_t ldx;
    int d, Kp;
    int split;          // 1: rows hold [bf16(x) | bf16(x - bf16(x))]
    __nv_bfloat16 *xb;  // n x Kp (x 2 when split)
};
struct TcCPrep {
    const double *c;    // k x d
    int64_t k, kpad;
    int d, Kp;
    int split;
    __nv_bfloat16 *cb;  // kpad x Kp (x 2 when split): -2 c
    __nv_bfloat16 *cbx; // kpad x 16: |c|^2 as bf16 hi, mid, lo, then zeros
    float *cn;          // kpad: |c|^2 in FP32 (for max |c|)
    unsigned *cmax_bits;
};

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_KB = 64;  // bf16 elements per 128-byte swizzle row
constexpr int TC_EPI_WARPS = 8;                   // 2 per TMEM lane quarter
constexpr int TC_EPI_GROUPS = TC_EPI_WARPS / 4;     // column groups per tile
constexpr int TC_MISC = 2048;                       // barriers, TMEM slot, merge buffer
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr int TC_KP_MAX = 128;                      // d <= 128
constexpr int TC_A_STAGE = TC_M * TC_KP_MAX * 2;    // bytes of one X tile stage
constexpr int TC_B_STAGE = TC_N * TC_KP_MAX * 2;    // bytes of one centre tile stage
// split-BF16 mode: tiles hold [hi | lo] (2 Kp columns); the same 192 KB is
// cut into larger X stages and smaller centre stages (N * Kp <= 8192)
constexpr int TC_A_STAGE_X3 = 2 * TC_A_STAGE;
constexpr int TC_B_STAGE_X3 = TC_B_STAGE / 2;
static_assert(TC_A_STAGE_X3 + TC_B_STAGE_X3 == TC_A_STAGE + TC_B_STAGE, "both modes share one layout size");
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcArgs {
    const TcInst *inst;
    const int2 *units;           // (instance, row tile); null: instance 0, unit = row tile
    int64_t nunits;
    int32_t *flag_rows;          // global rows whose argmin needs the FP64 decision
    unsigned long long *n_flag;
    int *err;
    int lg_ns;                   // log2 of the centre-tile ring's stages (1..3)
};

// three-input minimum
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Rigorous half-window of the BF16 path for one object.  The accumulator
// holds |c|^2 - 2 x_h.c_h summed by the tensor core: -2 c is exact in BF16,
// and |c|^2 enters as hi + mid + lo BF16 terms (within 2^-24 |c|^2) times one.
//   inputs rounded to bf16 (u_b = 2^-8):     2 (2 u_b + u_b^2) |x| cmax
//   |c|^2 split:                             2^-24 cmax^2
//   the tensor core's accumulation of the d + 3 products, bounded loosely
//   by (d + 19) 2^-21 of the sum of their magnitudes:
//                                            (d + 19) 2^-21 (2 |x| cmax + cmax^2)(1 + 2 u_b)
//   the FP64 reference's own error:          (d + 3) 2^-53 (|x| + cmax)^2
// times 1.01 for second-order terms.
__device__ __forceinline__ float window_bf16(float xn, float cmax, int d) {
    const float ub = 0.00390625f;
    const float xc = xn * cmax, c2 = cmax * cmax;
    const float e = 2.f * (2.f * ub + ub * ub) * xc + 5.9604645e-8f * c2 +
                    (float)(d + 19) * 4.76837158e-7f * (2.f * xc + c2) * (1.f + 2.f * ub);
    const float s = xn + cmax;
    const float e64 = (float)(d + 3) * 1.1102230e-16f * s * s;
    return 1.01f * (e + e64) + 1e-30f;
}

// Rigorous half-window of the split-BF16 path.  With x_h = bf16(x), x_l =
// bf16(x - x_h) (and the same for c), x.c - (x_h.c_h + x_l.c_h + x_h.c_l) =
// -(x - x_h - x_l).c_h - x_h.(c - c_h - c_l) + (x - x_h).(c - c_h), each
// term bounded by u_b^2 (1 + u_b) |x| |c|: input term 2 * 3 u_b^2 (1 + u_b)
// |x| cmax; the |c|^2 split 2^-24 cmax^2; the accumulation of 3d + 3
// products (3d + 19) 2^-21 (2 |x| cmax (1 + 4 u_b) + cmax^2 (1 + 2 u_b)); the
// FP64 reference term as in window_bf16; times 1.01.
__device__ __forceinline__ float window_bf16x3(float xn, float cmax, int d) {
    const float ub = 0.00390625f;
    const float xc = xn * cmax, c2 = cmax * cmax;
    const float e = 6.f * ub * ub * (1.f + ub) * xc + 5.9604645e-8f * c2 +
                    (float)(3 * d + 19) * 4.76837158e-7f * (2.f * xc * (1.f + 4.f * ub) + c2 * (1.f + 2.f * ub));
    const float s = xn + cmax;
    const float e64 = (float)(d + 3) * 1.1102230e-16f * s * s;
    return 1.01f * (e + e64) + 1e-30f;
}

// Running minimum of one warp's rows over NCH 32-column chunks of one
// accumulator tile (columns jb .. jb + 32 NCH - 1); the TMEM load of chunk
// ch + 1 is in flight while chunk ch is reduced.  Per row:
//   b1     the smallest value so far, found in the chunk saved in sv / sj
//   b2o    the smallest value outside that chunk
// A chunk with a new minimum is copied to sv (its index and second-smallest
// value are resolved once per row tile, see epi_resolve); any other chunk
// only lowers b2o.  So min(b2o, second smallest of sv) is exactly the
// runner-up over all columns.
template <int NCH>
__device__ __forceinline__ void epi_tile(uint32_t tbase, int64_t jb, float &b1, float &b2o, float (&sv)[32],
                                         int64_t &sj) {
    uint32_t ra[32], rb[32];
    tmem_ld32_async(tbase, ra);
    tmem_wait_ld();
#pragma unroll
    for (int ch = 0; ch < NCH; ch++) {
        if (ch + 1 < NCH) {
            if (ch & 1) tmem_ld32_async(tbase + (ch + 1) * 32, ra);
            else tmem_ld32_async(tbase + (ch + 1) * 32, rb);
        }
        const uint32_t *r = (ch & 1) ? rb : ra;
        float v[32];  // d' = |c|^2 - 2 x.c, straight from the accumulator
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
        float t11[11];
#pragma unroll
        for (int i = 0; i < 10; i++) t11[i] = min3f(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
        t11[10] = fminf(v[30], v[31]);
        const float tm = fminf(min3f(min3f(t11[0], t11[1], t11[2]), min3f(t11[3], t11[4], t11[5]),
                                     min3f(t11[6], t11[7], t11[8])),
                               fminf(t11[9], t11[10]));
        if (tm < b1) {
            b2o = fminf(b2o, b1);  // the old best chunk is now "outside"
            b1 = tm;
#pragma unroll
            for (int i = 0; i < 32; i++) sv[i] = v[i];
            sj = jb + ch * 32;
        } else {
            b2o = fminf(b2o, tm);
        }
        if (ch + 1 < NCH) tmem_wait_ld();
    }
}

// Index (first position) of the minimum in the saved chunk and the exact
// runner-up over all columns.
__device__ __forceinline__ void epi_resolve(float b1, float b2o, const float (&sv)[32], int64_t sj, float &b2,
                                            int &i1) {
    if (sj < 0) {  // no finite value at all
        b2 = b2o;
        i1 = 0x7FFFFFFF;
        return;
    }
    int idx = 31;
#pragma unroll
    for (int i = 31; i >= 0; i--)
        if (sv[i] == b1) idx = i;
    float m2 = FLT_MAX;
#pragma unroll
    for (int i = 0; i < 32; i++) m2 = fminf(m2, i == idx ? FLT_MAX : sv[i]);
    b2 = fminf(b2o, m2);
    i1 = (int)(sj + idx);
}

// SPLIT = false: S = x_h . c_h, one BF16 product per element (window_bf16).
// SPLIT = true: x = x_h + x_l and c = c_h + c_l in BF16 pairs, S = x_h . c_h +
// x_l . c_h + x_h . c_l: three MMAs per k-step into the same accumulator
// (window_bf16x3, ~100x narrower).
template <bool SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_assign_tc(const __grid_constant__ TcArgs A) {
    constexpr int A_ST = SPLIT ? TC_A_STAGE_X3 : TC_A_STAGE;
    constexpr int B_ST = SPLIT ? TC_B_STAGE_X3 : TC_B_STAGE;
    constexpr int KW = SPLIT ? 2 : 1;  // stored column blocks per k-block
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA0 = base, *sB0 = base + 2 * A_ST;
    uint64_t *bars = (uint64_t *)(base + 2 * TC_A_STAGE + 2 * TC_B_STAGE);
    uint64_t *full_a = bars, *empty_a = bars + 2, *full_acc = bars + 4, *empty_acc = bars + 6;
    uint64_t *done_bar = bars + 8, *full_b = bars + 9, *empty_b = bars + 17;  // B ring: up to 8 stages
    uint32_t *tmem_slot = (uint32_t *)(bars + 25);
    // the centre-tile ring: the same bytes cut into NS stages (narrower tiles,
    // more stages in flight)
    const int NS = 1 << A.lg_ns;
    const int BSTR = 2 * B_ST / NS, XSTR = 2 * TC_N * 32 / NS;
    float *mrg = (float *)(bars + 32);  // [groups-1][128][3] results of column groups 1..
    // |c|^2 columns: an all-ones X block (128 x 16) and per stage the centres'
    // (hi, mid, lo, 0...) rows (N x 16), 32-byte swizzled; one extra K = 16
    // step adds |c|^2 to every accumulator column
    uint8_t *sOnes = base + 2 * TC_A_STAGE + 2 * TC_B_STAGE + TC_MISC;  // 4 KB
    uint8_t *sX0 = sOnes + TC_M * 32;                                   // [2][TC_N * 32]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(&full_a[i], 1);
            mbar_init(&empty_a[i], 1);
            mbar_init(&full_acc[i], 1);
            mbar_init(&empty_acc[i], TC_EPI_WARPS);
        }
        for (int i = 0; i < 8; i++) {
            mbar_init(&full_b[i], 1);
            mbar_init(&empty_b[i], 1);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the all-ones block (1.0 in BF16 everywhere, so its swizzle is moot)
    for (int e = threadIdx.x; e < TC_M * 32 / 4; e += blockDim.x)
        reinterpret_cast<uint32_t *>(sOnes)[e] = 0x3F803F80u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    // Every role walks the same unit sequence (unit u = blockIdx.x + j *
    // gridDim.x); an instance's Kp, N and centre-tile count fix the per-unit
    // copy sizes, MMA shape and epilogue width.
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint64_t ct = 0;
            uint32_t issued_b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            bool ok = true;
            int64_t it = 0;
            for (int64_t u = blockIdx.x; u < A.nunits && ok; u += gridDim.x, it++) {
                const int2 un = A.units ? A.units[u] : make_int2(0, (int)u);
                const TcInst &I = A.inst[un.x];
                const int nkb = KW * I.Kp / TC_KB, N = I.N;  // stored k-blocks
                const uint32_t a_bytes = (uint32_t)TC_M * KW * I.Kp * 2, b_bytes = (uint32_t)N * KW * I.Kp * 2;
                const int ab = (int)(it & 1);
                const uint32_t ua = (uint32_t)(it >> 1);
                if (!(ok = mbar_wait(&empty_a[ab], (ua & 1) ^ 1, A.err))) break;
                mbar_expect_tx(&full_a[ab], a_bytes);
                for (int kb = 0; kb < nkb; kb++)
                    tma_load_2d(su32(sA0 + ab * A_ST + kb * TC_M * 128), &I.tmA, kb * TC_KB, un.y * TC_M,
                                &full_a[ab]);
                for (int c = 0; c < I.ntiles_c; c++, ct++) {
                    const int s = (int)(ct & (uint64_t)(NS - 1));
                    const uint32_t uu = (uint32_t)(ct >> A.lg_ns);
                    if (!(ok = mbar_wait(&empty_b[s], (uu & 1) ^ 1, A.err))) break;
                    mbar_expect_tx(&full_b[s], b_bytes + (uint32_t)N * 32);
                    for (int kb = 0; kb < nkb; kb++)
                        tma_load_2d(su32(sB0 + s * BSTR + kb * N * 128), &I.tmB, kb * TC_KB, c * N, &full_b[s]);
                    tma_load_2d(su32(sX0 + s * XSTR), &I.tmX, 0, c * N, &full_b[s]);
                    issued_b[s] = uu + 1;
                }
            }
            // drain: every centre-tile copy this thread issued has landed
            for (int s = 0; s < NS; s++)
                if (issued_b[s]) mbar_wait(&full_b[s], (issued_b[s] - 1) & 1, A.err, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint64_t ct = 0;
            bool ok = true;
            int64_t it = 0;
            for (int64_t u = blockIdx.x; u < A.nunits && ok; u += gridDim.x, it++) {
                const int2 un = A.units ? A.units[u] : make_int2(0, (int)u);
                const TcInst &I = A.inst[un.x];
                const int nkb = I.Kp / TC_KB, N = I.N;  // logical k-blocks
                const uint32_t idesc = idesc_bf16(TC_M, N);
                const int ab = (int)(it & 1);
                const uint32_t ua = (uint32_t)(it >> 1);
                if (!(ok = mbar_wait(&full_a[ab], ua & 1, A.err))) break;
                const uint32_t a_base = su32(sA0 + ab * A_ST);
                for (int c = 0; c < I.ntiles_c; c++, ct++) {
                    const int sb = (int)(ct & (uint64_t)(NS - 1));  // centre-tile stage
                    const uint32_t ub = (uint32_t)(ct >> A.lg_ns);
                    const int s = (int)(ct & 1);                     // accumulator buffer
                    const uint32_t uu = (uint32_t)(ct >> 1);
                    if (!(ok = mbar_wait(&full_b[sb], ub & 1, A.err))) break;
                    if (!(ok = mbar_wait(&empty_acc[s], (uu & 1) ^ 1, A.err))) break;
                    fence_after();
                    const uint32_t b_base = su32(sB0 + sb * BSTR);
                    const uint32_t dtm = tmem + (uint32_t)(s * TC_N);
                    for (int kb = 0; kb < nkb; kb++)
#pragma unroll
                        for (int ks = 0; ks < TC_KB / 16; ks++) {
                            const uint32_t ao = kb * TC_M * 128 + ks * 32, bo = kb * N * 128 + ks * 32;
                            mma_bf16(dtm, sdesc(a_base + ao), sdesc(b_base + bo), idesc, (kb | ks) != 0);
                            if (SPLIT) {
                                // x_l . c_h and x_h . c_l: the lo halves sit nkb k-blocks on
                                mma_bf16(dtm, sdesc(a_base + ao + nkb * TC_M * 128), sdesc(b_base + bo), idesc, 1);
                                mma_bf16(dtm, sdesc(a_base + ao), sdesc(b_base + bo + nkb * N * 128), idesc, 1);
                            }
                        }
                    // + |c|^2: ones (128 x 16) times the centres' (hi, mid, lo, 0...)
                    mma_bf16(dtm, sdesc32(su32(sOnes)), sdesc32(su32(sX0 + sb * XSTR)), idesc, 1);
                    mma_commit(&empty_b[sb]);
                    mma_commit(&full_acc[s]);
                }
                mma_commit(&empty_a[ab]);
            }
            // drain: all MMAs this thread issued have completed
            mma_commit(done_bar);
            mbar_wait(done_bar, 0, A.err, true);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int ew = warp - 2;
        const int q = warp & 3;     // TMEM lane quarter this warp may access
        const int h = ew >> 2;      // column group
        const int rloc = 32 * q + lane;
        uint64_t ct = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < A.nunits; u += gridDim.x) {
            const int2 un = A.units ? A.units[u] : make_int2(0, (int)u);
            const TcInst &I = A.inst[un.x];
            const int N = I.N;
            const int gcols = N / TC_EPI_GROUPS;  // columns of this warp's group
            const int nch = gcols / 32;           // 32-column chunks (1, 2 or 4)
            const int64_t row = (int64_t)un.y * TC_M + rloc;
            const float xn = row < I.n ? I.xnorm[row] : 0.f;
            const float cmax = sqrtf(__uint_as_float(*I.cmax_bits)) * (1.f + 1e-5f);
            const float W = 2.f * (SPLIT ? window_bf16x3(xn, cmax, I.d) : window_bf16(xn, cmax, I.d));
            const float Wc = W * (1.f + 1e-6f);
            float b1 = FLT_MAX, b2o = FLT_MAX, sv[32];
            int64_t sj = -1;
            for (int c = 0; c < I.ntiles_c; c++, ct++) {
                const int s = (int)(ct & 1);
                const uint32_t uu = (uint32_t)(ct >> 1);
                int w_ok = 0;
                if (lane == 0 && ok) w_ok = mbar_wait(&full_acc[s], uu & 1, A.err);
                w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
                ok = ok && w_ok;
                if (ok) {
                    fence_after();
                    const uint32_t tbase = tmem + (uint32_t)(s * TC_N + h * gcols) + ((uint32_t)(32 * q) << 16);
                    const int64_t jb = (int64_t)c * N + h * gcols;
                    if (nch == 4) epi_tile<4>(tbase, jb, b1, b2o, sv, sj);
                    else if (nch == 2) epi_tile<2>(tbase, jb, b1, b2o, sv, sj);
                    else epi_tile<1>(tbase, jb, b1, b2o, sv, sj);
                    fence_before();
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty_acc[s]);
            }
            float b2;
            int i1;
            epi_resolve(b1, b2o, sv, sj, b2, i1);
            // merge the column groups of each row
            asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_EPI_WARPS) : "memory");
            if (h > 0) {
                float *m = mrg + ((h - 1) * TC_M + rloc) * 3;
                m[0] = b1;
                m[1] = b2;
                m[2] = __int_as_float(i1);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_EPI_WARPS) : "memory");
            if (h == 0 && row < I.n && ok) {
#pragma unroll
                for (int g = 1; g < TC_EPI_GROUPS; g++) {
                    const float *m = mrg + ((g - 1) * TC_M + rloc) * 3;
                    const float ob1 = m[0], ob2 = m[1];
                    const int oi1 = __float_as_int(m[2]);
                    // equal best values leave b2 == b1: the row is then
                    // flagged and decided in FP64, so the index is moot
                    float nb2;
                    if (ob1 < b1) {
                        nb2 = fminf(b1, fminf(b2, ob2));
                        b1 = ob1;
                        i1 = oi1;
                    } else {
                        nb2 = fminf(ob1, fminf(b2, ob2));
                    }
                    b2 = nb2;
                }
                const bool valid = i1 != 0x7FFFFFFF;
                I.labels[row] = valid ? i1 : -1;
                const bool sure = valid && (I.k == 1 || b2 - b1 > Wc);
                if (!sure) {
                    const unsigned long long qq = atomicAdd(A.n_flag, 1ull);
                    A.flag_rows[qq] = (int32_t)(I.row_base + row);
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_EPI_WARPS) : "memory");
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// X -> BF16 K-major [n][Kp] (zero padded) and an upper bound of |x| per row;
// warp per global row r of instance find_inst(row_off, r); xnorm is global.
// A lane converts 4 consecutive columns at a time (float4 loads, 8-byte
// stores) when the row is 16-byte aligned.
__global__ void k_x_to_bf16(const TcXPrep *__restrict__ X, const int64_t *__restrict__ row_off, int count, int64_t N,
                            float *__restrict__ xnorm) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // one instance: rows strided over the warps; several: a contiguous range
    // of rows per warp, the instance looked up again only when the range
    // crosses into the next one
    const bool one = count == 1;
    const int64_t per = one ? 0 : (N + nw - 1) / nw;
    const int64_t rbeg = one ? warp : warp * per, rend = one ? N : min(N, rbeg + per), rstep = one ? nw : 1;
    int ii = 0;
    int64_t ilo = 0, ihi = one ? N : -1;
    for (int64_t r = rbeg; r < rend; r += rstep) {
        if (r < ilo || r >= ihi) {
            ii = find_inst(row_off, count, r);
            ilo = row_off[ii];
            ihi = row_off[ii + 1];
        }
        const TcXPrep &P = X[ii];
        const int64_t i = r - row_off[ii];
        const int W = P.split ? 2 * P.Kp : P.Kp;
        const float *xr = P.x + i * P.ldx;
        __nv_bfloat16 *hb = P.xb + i * W;
        float s = 0.f;
        if (((P.ldx & 3) == 0) && ((P.d & 3) == 0) && (((uintptr_t)P.x & 15) == 0)) {
            for (int t = 4 * lane; t < P.Kp; t += 128) {
                const float4 v = t < P.d ? *reinterpret_cast<const float4 *>(xr + t) : make_float4(0.f, 0.f, 0.f, 0.f);
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
                uint2 hv;
                hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                *reinterpret_cast<uint2 *>(hb + t) = hv;
                if (P.split) {
                    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);  // differences exact
                    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
                    uint2 lv;
                    lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                    lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                    *reinterpret_cast<uint2 *>(hb + P.Kp + t) = lv;
                }
                s = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, s))));
            }
        } else {
            for (int t = lane; t < P.Kp; t += 32) {
                const float v = t < P.d ? xr[t] : 0.f;
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                hb[t] = h;
                if (P.split) hb[P.Kp + t] = __float2bfloat16_rn(v - __bfloat162float(h));  // v - h exact
                s = fmaf(v, v, s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) xnorm[r] = sqrtf(s) * (1.f + 1.0e-3f);
    }
}

// centres -> BF16 [kpad][Kp], |c|^2 (+inf for padding) and the max of |c|^2
// over real centres; thread per global padded centre e of instance
// find_inst(kpad_off, e)
__global__ void k_c_to_bf16(const TcCPrep *__restrict__ C, const int64_t *__restrict__ kpad_off, int count,
                            int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ii = find_inst(kpad_off, count, e);
        const TcCPrep &P = C[ii];
        const int64_t j = e - kpad_off[ii];
        const int W = P.split ? 2 * P.Kp : P.Kp;
        double s = 0.0;
        for (int t = 0; t < P.Kp; t++) {
            // -2 c: scaling by a power of two is exact in BF16
            const double v = (j < P.k && t < P.d) ? P.c[j * P.d + t] : 0.0;
            const __nv_bfloat16 h = __double2bfloat16(-2.0 * v);
            P.cb[j * W + t] = h;
            if (P.split) P.cb[j * W + P.Kp + t] = __double2bfloat16(-2.0 * v - (double)__bfloat162float(h));  // exact
            s += v * v;
        }
        // |c|^2 = hi + mid + lo in BF16 (within 2^-24 |c|^2); padding: +inf,
        // which never wins
        __nv_bfloat16 *xr = P.cbx + j * 16;
        if (j < P.k) {
            const __nv_bfloat16 h = __double2bfloat16(s);
            const double r1 = s - (double)__bfloat162float(h);
            const __nv_bfloat16 m = __double2bfloat16(r1);
            const double r2 = r1 - (double)__bfloat162float(m);
            xr[0] = h;
            xr[1] = m;
            xr[2] = __double2bfloat16(r2);
        } else {
            xr[0] = __ushort_as_bfloat16((unsigned short)0x7F80);
            xr[1] = __ushort_as_bfloat16((unsigned short)0);
            xr[2] = __ushort_as_bfloat16((unsigned short)0);
        }
        for (int t = 3; t < 16; t++) xr[t] = __ushort_as_bfloat16((unsigned short)0);
        const float f = (float)s;
        P.cn[j] = j < P.k ? f : __int_as_float(0x7f800000);
        if (j < P.k) atomicMax(P.cmax_bits, __float_as_uint(f));  // non-negative floats order as uints
    }
}

constexpr int TC_TILES[3] = {64, 128, 256};

}  // namespace

struct TcPlan::Impl {
    std::vector<TcInst> inst;      // host copy (tensor maps for the chosen N)
    std::vector<TcXPrep> xp;
    std::vector<TcCPrep> cp;
    std::vector<int64_t> kpad_off;
};

namespace {

template <class T>
geek_status plan_alloc(geek_ctx *ctx, Scratch *scr, std::vector<void *> &owned, T **p, size_t count) {
    if (scr) return scr->alloc(p, count);
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
    }
    owned.push_back(q);
    *p = (T *)q;
    return GEEK_OK;
}

// TcInst of instance i for tile width N (tensor maps re-encoded)
geek_status make_inst(geek_ctx *ctx, const TcPlan &P, int i, int N, TcInst *out) {
    const TcPlanInst &I = P.desc[i];
    const int Kp = I.d <= 64 ? 64 : 128;
    TcInst T;
    memset(&T, 0, sizeof T);
    const TcXPrep &xp = P.impl->xp[i];
    const TcCPrep &cp = P.impl->cp[i];
    const int Kst = I.split ? 2 * Kp : Kp;  // stored columns
    if (I.split && N * Kp > 8192)
        return set_error(ctx, GEEK_ERR_INVALID, "split-BF16 tiles need N * Kp <= 8192 (N %d, Kp %d)", N, Kp);
    if (I.n > 0) GK_TRY(encode_bf16_2d(ctx, &T.tmA, xp.xb, Kst, I.n, TC_KB, TC_M));
    if (I.k > 0) GK_TRY(encode_bf16_2d(ctx, &T.tmB, cp.cb, Kst, cp.kpad, TC_KB, N));
    if (I.k > 0) GK_TRY(encode_bf16_2d(ctx, &T.tmX, cp.cbx, 16, cp.kpad, 16, N, CU_TENSOR_MAP_SWIZZLE_32B));
    T.xnorm = P.xnorm + I.row_base;
    T.cmax_bits = cp.cmax_bits;
    T.labels = I.labels;
    T.n = I.n;
    T.k = I.k;
    T.row_base = I.row_base;
    T.ntiles_c = (int)ceil_div(I.k, N);
    T.Kp = Kp;
    T.d = I.d;
    T.N = N;
    *out = T;
    return GEEK_OK;
}

// units of the listed instances in one mode (split or not), longest first
// (LPT order over the CTAs)
void make_units(const TcPlan &P, const std::vector<int> &which, int split, std::vector<int2> &units) {
    std::vector<std::pair<int64_t, int>> cost;
    for (int i : which) {
        const TcInst &T = P.impl->inst[i];
        if (T.n <= 0 || T.k <= 0 || P.desc[i].split != split) continue;
        cost.push_back({(int64_t)T.ntiles_c * T.N * T.Kp * (split ? 3 : 1) + 2048, i});
    }
    std::stable_sort(cost.begin(), cost.end(), [](const std::pair<int64_t, int> &a, const std::pair<int64_t, int> &b) {
        return a.first > b.first;
    });
    units.clear();
    for (auto &c : cost) {
        const int64_t nt = ceil_div(P.impl->inst[c.second].n, TC_M);
        for (int64_t r = 0; r < nt; r++) units.push_back(make_int2(c.second, (int)r));
    }
}

size_t tc_smem() {
    static_assert(32 * 8 + (TC_EPI_GROUPS - 1) * TC_M * 3 * 4 <= TC_MISC, "misc region too small");
    // tile stages + barriers / TMEM slot / merge buffer + |c|^2 ring + alignment
    // tile stages + barriers / TMEM slot / merge buffer + ones block + two
    // |c|^2 stages + alignment
    return 1024 + 2 * (size_t)TC_A_STAGE + 2 * (size_t)TC_B_STAGE + TC_MISC + TC_M * 32 + 2 * TC_N * 32;
}

}  // namespace

int tc_tile_candidates(const int **tiles) {
    *tiles = TC_TILES;
    return 3;
}

geek_status tc_plan_build(geek_ctx *ctx, Scratch *scr, const std::vector<TcPlanInst> &desc, TcPlan *P,
                          cudaStream_t st) {
    P->impl = new TcPlan::Impl();
    P->desc = desc;
    const int count = (int)desc.size();
    P->count = count;
    auto &im = *P->impl;
    std::vector<int64_t> row_off(count + 1, 0);
    im.kpad_off.assign(count + 1, 0);
    int64_t xb_total = 0, cb_total = 0;
    for (int i = 0; i < count; i++) {
        const TcPlanInst &I = desc[i];
        if (I.d > TC_KP_MAX || I.d <= 0)
            return set_error(ctx, GEEK_ERR_UNSUPPORTED, "BF16 tensor-core assignment supports 1 <= d <= 128");
        if (I.N != 64 && I.N != 128 && I.N != 256) return set_error(ctx, GEEK_ERR_INVALID, "tile N must be 64/128/256");
        const int Kp = I.d <= 64 ? 64 : 128;
        // room for the split layout whenever a plan may switch modes
        const int Kst = (I.split || P->allow_split) ? 2 * Kp : Kp;
        row_off[i + 1] = row_off[i] + I.n;
        // padding to a multiple of 256 serves every tile width
        im.kpad_off[i + 1] = im.kpad_off[i] + ceil_div(I.k, TC_N) * TC_N;
        xb_total += I.n * Kst;
        cb_total += ceil_div(I.k, TC_N) * TC_N * Kst;
    }
    P->N_total = row_off[count];
    P->kpad_total = im.kpad_off[count];
    auto &own = P->owned;
    __nv_bfloat16 *xb, *cb, *cbx;
    float *cn;
    unsigned *cmax_bits;
    GK_TRY(plan_alloc(ctx, scr, own, &xb, (size_t)std::max<int64_t>(xb_total, 1)));
    GK_TRY(plan_alloc(ctx, scr, own, &cb, (size_t)std::max<int64_t>(cb_total, 1)));
    GK_TRY(plan_alloc(ctx, scr, own, &cbx, (size_t)std::max<int64_t>(im.kpad_off[count] * 16, 1)));
    GK_TRY(plan_alloc(ctx, scr, own, &P->xnorm, (size_t)std::max<int64_t>(P->N_total, 1)));
    GK_TRY(plan_alloc(ctx, scr, own, &cn, (size_t)std::max<int64_t>(P->kpad_total, 1)));
    GK_TRY(plan_alloc(ctx, scr, own, &cmax_bits, (size_t)count));
    GK_TRY(plan_alloc(ctx, scr, own, &P->row_off, (size_t)count + 1));
    GK_TRY(plan_alloc(ctx, scr, own, &P->kpad_off_dev, (size_t)count + 1));
    GK_TRY(plan_alloc(ctx, scr, own, &P->xprep, (size_t)count));
    GK_TRY(plan_alloc(ctx, scr, own, &P->cprep, (size_t)count));
    GK_TRY(plan_alloc(ctx, scr, own, &P->inst, (size_t)count));
    GK_TRY(plan_alloc(ctx, scr, own, &P->err, 1));
    P->cmax_bits = cmax_bits;
    im.xp.resize(count);
    im.cp.resize(count);
    int64_t xo = 0, co = 0;
    for (int i = 0; i < count; i++) {
        const TcPlanInst &I = desc[i];
        const int Kp = I.d <= 64 ? 64 : 128;
        const int Kst = (I.split || P->allow_split) ? 2 * Kp : Kp;
        im.xp[i] = TcXPrep{I.x, I.ldx, I.d, Kp, I.split, xb + xo};
        const int64_t kpad = im.kpad_off[i + 1] - im.kpad_off[i];
        im.cp[i] = TcCPrep{I.centres, I.k, kpad, I.d, Kp, I.split, cb + co, cbx + im.kpad_off[i] * 16,
                           cn + im.kpad_off[i], cmax_bits + i};
        xo += I.n * Kst;
        co += kpad * Kst;
    }
    im.inst.resize(count);
    for (int i = 0; i < count; i++) GK_TRY(make_inst(ctx, *P, i, desc[i].N, &im.inst[i]));
    GK_TRY(plan_alloc(ctx, scr, own, &P->units, (size_t)std::max<int64_t>(ceil_div(P->N_total, TC_M) + count, 1)));
    GK_CUDA(ctx, cudaMemcpyAsync(P->row_off, row_off.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaMemcpyAsync(P->kpad_off_dev, im.kpad_off.data(), sizeof(int64_t) * (count + 1),
                                 cudaMemcpyHostToDevice, st));
    GK_TRY(tc_plan_upload(ctx, P, st));
    GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem()));
    GK_CUDA(ctx, cudaFuncSetAttribute(k_assign_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem()));
    return GEEK_OK;
}

// Uploads the descriptors and unit lists of the current modes and tiles:
// units[0, nunits) run in BF16, units[nunits, nunits + nunits_x3) in
// split-BF16.
geek_status tc_plan_upload(geek_ctx *ctx, TcPlan *P, cudaStream_t st) {
    auto &im = *P->impl;
    const int count = P->count;
    for (int i = 0; i < count; i++) {
        im.xp[i].split = P->desc[i].split;
        im.cp[i].split = P->desc[i].split;
    }
    std::vector<int> all(count);
    for (int i = 0; i < count; i++) all[i] = i;
    std::vector<int2> u0, u1;
    make_units(*P, all, 0, u0);
    make_units(*P, all, 1, u1);
    P->nunits = (int64_t)u0.size();
    P->nunits_x3 = (int64_t)u1.size();
    u0.insert(u0.end(), u1.begin(), u1.end());
    GK_CUDA(ctx, cudaMemcpyAsync(P->xprep, im.xp.data(), sizeof(TcXPrep) * count, cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaMemcpyAsync(P->cprep, im.cp.data(), sizeof(TcCPrep) * count, cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaMemcpyAsync(P->inst, im.inst.data(), sizeof(TcInst) * count, cudaMemcpyHostToDevice, st));
    if (!u0.empty())
        GK_CUDA(ctx, cudaMemcpyAsync(P->units, u0.data(), sizeof(int2) * u0.size(), cudaMemcpyHostToDevice, st));
    // the host vectors are pageable: the copies have read them on return
    return GEEK_OK;
}

// Conversions of X and the centres (BF16 or split-BF16 pairs, norms, the
// max of |c|^2).  No host synchronisation.
geek_status tc_plan_convert(geek_ctx *ctx, const TcPlan &P, cudaStream_t st) {
    const int count = P.count;
    GK_CUDA(ctx, cudaMemsetAsync(P.err, 0, sizeof(int), st));
    GK_CUDA(ctx, cudaMemsetAsync(P.cmax_bits, 0, sizeof(unsigned) * count, st));
    if (P.N_total > 0) {
        GK_COUNT();
        k_x_to_bf16<<<grid_for(P.N_total * 32, 256, ctx->num_sms), 256, 0, st>>>(P.xprep, P.row_off, count,
                                                                                 P.N_total, P.xnorm);
    }
    if (P.kpad_total > 0) {
        GK_COUNT();
        k_c_to_bf16<<<grid_for(P.kpad_total, 128, ctx->num_sms), 128, 0, st>>>(P.cprep, P.kpad_off_dev, count,
                                                                               P.kpad_total);
    }
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

namespace {

// log2 of the centre-tile ring's stages for the instances of one mode in a
// launch: the widest stage among them fixes the stage size; the ring's bytes
// are cut into as many stages as fit (2 .. 8). Two regions are cut: the
// centre tiles (N x Kp BF16, twice that when split) and the |c|^2 rows
// (N x 32 bytes out of 2 * TC_N * 32), so both bound the stage count.
int ring_lg(const TcPlan &P, const std::vector<int> *which, int split) {
    int64_t mx = 0, nmax = 0;
    auto consider = [&](int i) {
        const TcPlanInst &I = P.desc[i];
        if ((I.split != 0) != (split != 0)) return;
        const int64_t Kp = I.d <= 64 ? 64 : 128;
        mx = std::max<int64_t>(mx, (int64_t)I.N * Kp * 2 * (split ? 2 : 1));
        nmax = std::max<int64_t>(nmax, (int64_t)I.N);
    };
    if (which)
        for (int i : *which) consider(i);
    else
        for (int i = 0; i < P.count; i++) consider(i);
    const int64_t ring = 2 * (int64_t)(split ? TC_B_STAGE_X3 : TC_B_STAGE);
    int lg = 1;
    const int64_t xring = 2 * (int64_t)TC_N * 32;
    while (lg < 3 && mx > 0 && (ring >> (lg + 1)) >= mx && (xring >> (lg + 1)) >= nmax * 32) lg++;
    return lg;
}

geek_status launch_units(geek_ctx *ctx, const TcInst *inst, const int2 *units, int64_t n0, int64_t n1,
                         int32_t *flag_rows, unsigned long long *n_flag, int *err, double work, int lg0, int lg1,
                         cudaStream_t st) {
    TcArgs A;
    A.inst = inst;
    A.flag_rows = flag_rows;
    A.n_flag = n_flag;
    A.err = err;
    EvTimer tk(ctx, "kernel.assign_tc", st);
    tk.work = work;
    if (n0 > 0) {
        A.units = units;
        A.nunits = n0;
        A.lg_ns = lg0;
        GK_COUNT();
        k_assign_tc<false><<<(int)std::min<int64_t>(n0, ctx->num_sms), TC_THREADS, tc_smem(), st>>>(A);
    }
    if (n1 > 0) {
        A.units = units + n0;
        A.nunits = n1;
        A.lg_ns = lg1;
        GK_COUNT();
        k_assign_tc<true><<<(int)std::min<int64_t>(n1, ctx->num_sms), TC_THREADS, tc_smem(), st>>>(A);
    }
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

}  // namespace

// The persistent tcgen05 passes (BF16 units, then split-BF16 units) after
// tc_plan_convert; flagged rows are appended to flag_rows / n_flag (zeroed
// by the caller).
geek_status tc_plan_launch(geek_ctx *ctx, const TcPlan &P, int32_t *flag_rows, unsigned long long *n_flag,
                           cudaStream_t st) {
    double work = 0.0;
    for (const TcPlanInst &I : P.desc) work += 2.0 * (double)I.n * (double)I.k * (double)I.d;
    return launch_units(ctx, P.inst, P.units, P.nunits, P.nunits_x3, flag_rows, n_flag, P.err, work,
                        ring_lg(P, nullptr, 0), ring_lg(P, nullptr, 1), st);
}

geek_status tc_plan_enqueue(geek_ctx *ctx, const TcPlan &P, int32_t *flag_rows, unsigned long long *n_flag,
                            cudaStream_t st) {
    GK_TRY(tc_plan_convert(ctx, P, st));
    return tc_plan_launch(ctx, P, flag_rows, n_flag, st);
}

// Sets every instance's tile width and mode (descriptors re-encoded, units
// rebuilt).  The next tc_plan_convert writes the matching layouts.
geek_status tc_plan_set_modes(geek_ctx *ctx, TcPlan *P, const std::vector<int> &N, const std::vector<int> &split,
                              cudaStream_t st) {
    for (int i = 0; i < P->count; i++) {
        if (split[i] && !P->allow_split && !P->desc[i].split)
            return set_error(ctx, GEEK_ERR_INVALID, "plan was built without room for split-BF16");
        P->desc[i].N = N[i];
        P->desc[i].split = split[i];
        GK_TRY(make_inst(ctx, *P, i, N[i], &P->impl->inst[i]));
    }
    return tc_plan_upload(ctx, P, st);
}

// Launches the tcgen05 pass over the units of `which` only, with tile width
// N and mode `split` for those instances (their layouts must match: run
// tc_plan_convert after tc_plan_set_modes).  Uses the plan's scratch
// descriptor table; writes labels and flags of those rows.  No host sync.
geek_status tc_plan_launch_subset(geek_ctx *ctx, TcPlan *P, const std::vector<int> &which, int32_t *flag_rows,
                                  unsigned long long *n_flag, cudaStream_t st) {
    auto &im = *P->impl;
    std::vector<int2> u0, u1;
    make_units(*P, which, 0, u0);
    make_units(*P, which, 1, u1);
    const int64_t n0 = (int64_t)u0.size(), n1 = (int64_t)u1.size();
    u0.insert(u0.end(), u1.begin(), u1.end());
    if (u0.empty()) return GEEK_OK;
    if (!P->tune_units || P->tune_cap < (int64_t)u0.size()) {
        if (P->tune_units) cudaFree(P->tune_units);
        P->tune_units = nullptr;
        P->tune_cap = 0;
        if (cudaMalloc((void **)&P->tune_units, sizeof(int2) * u0.size()) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, GEEK_ERR_NOMEM, "autotune unit list");
        }
        P->tune_cap = (int64_t)u0.size();
    }
    GK_CUDA(ctx, cudaMemcpyAsync(P->tune_units, u0.data(), sizeof(int2) * u0.size(), cudaMemcpyHostToDevice, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));  // u0 is pageable and about to go out of scope
    (void)im;
    return launch_units(ctx, P->inst, P->tune_units, n0, n1, flag_rows, n_flag, P->err, 0.0, ring_lg(*P, &which, 0),
                        ring_lg(*P, &which, 1), st);
}

geek_status tc_plan_check(geek_ctx *ctx, const TcPlan &P, cudaStream_t st) {
    int h_err = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&h_err, P.err, sizeof h_err, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_err) return set_error(ctx, (geek_status)h_err, "tensor-core assignment: a pipeline wait timed out");
    return GEEK_OK;
}

void tc_plan_free(TcPlan *P) {
    for (void *p : P->owned) cudaFree(p);
    P->owned.clear();
    if (P->tune_units) cudaFree(P->tune_units);
    P->tune_units = nullptr;
    P->tune_cap = 0;
    delete P->impl;
    P->impl = nullptr;
}

// BF16 (split = 0) or split-BF16 (split = 1) tcgen05 pass of one data set:
// labels for every object, flagged rows appended to flag_rows / n_flag for
// the FP64 decision.  d <= 128.
geek_status assign_tc_bf16(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                           const double *centres, int64_t k, int split, int32_t *labels, int32_t *flag_rows,
                           unsigned long long *n_flag, cudaStream_t st) {
    if (d > 128) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "BF16 tensor-core assignment supports d <= 128");
    TcPlan P;
    std::vector<TcPlanInst> one(1);
    // BF16: N = 256 (two stages; 128-wide tiles read A from shared memory
    // twice as often per flop and measured ~60% slower at d = 128).  Split:
    // the widest tile whose hi|lo stage fits
    const int N = split ? (d <= 64 ? 128 : 64) : TC_N;
    one[0] = TcPlanInst{x, ldx, n, d, centres, k, labels, 0, N, split};
    struct Free {
        TcPlan *p;
        ~Free() { tc_plan_free(p); }
    } fr{&P};
    GK_TRY(tc_plan_build(ctx, &scr, one, &P, st));
    GK_TRY(tc_plan_enqueue(ctx, P, flag_rows, n_flag, st));
    return tc_plan_check(ctx, P, st);
}
