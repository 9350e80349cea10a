// Dense projection P = X A^T on the 5th-generation tensor cores (tcgen05),
// fused with the E2LSH / SRP epilogue of Sect. 3.1 (Remarks): code =
// floor((a.x + b) / w) or the sign bit [a.x >= 0], exact after the boundary
// recheck of the elements whose error window straddles a cell edge.
//
// Three-term BF16 split.  x = x1 + x2 + x3 + rx with x1 = bf16(x), x2 =
// bf16(x - x1), x3 = bf16(x - x1 - x2) (both differences exact in FP32) and
// |rx| <= 2^-24 |x|; the same for a.  Every BF16 x BF16 product is exact.
// The six products of order <= 4 go to two TMEM accumulators:
//   P = sum_j a1 x1                      (the large term)
//   Q = sum_j a1 x2 + a2 x1 + a1 x3 + a2 x2 + a3 x1   (about 2^-7 of P)
// so the error of the large accumulation does not grow with the number of
// small products, and v = fl(P + Q).
//
// Rigorous window (S = sum_j |a_j x_j| <= |a| |x|):
//   dropped terms a2 x3, a3 x2, a3 x3 and the split residues:  2^-22 S
//   tensor-core accumulation, modelled per MMA instruction (16 products plus
//   the accumulator) as at most 2^-20 (|D_in| + sum |products|):
//       P: n_k 2^-20 S(1 + 2^-8)^2,  Q: 5 n_k 2^-20 (0.0079 S)
//     (n_k = k-steps of 16 columns holding data)
//   the final FP32 add P + Q:                                   2^-24 S
//   the FP64 reference's own error:                             d 2^-53 S
// times 1.01; with d = 128 this is 8.4e-6 |a||x|, about the FP32 SIMT
// path's gamma_d |a||x| (7.7e-6).  The per-instruction bound is a model of
// the tensor core's FP32 accumulation (products exact, aligned sum of one
// instruction's terms with at most a few units of 2^-23 of their magnitude
// lost), taken with a factor of two beyond that.
//
// Persistent kernel, one CTA per SM, 22 warps:
//   warp 0      TMA producer: the split image of A once (bulk copy), then X
//               in FP32 boxes of 128 rows x 32 columns (3-stage ring)
//   warp 1      MMA issuer: per k-step six tcgen05.mma (M = 128, N = F
//               padded to 32) into P and Q, double-buffered in TMEM
//   warps 2-13  epilogue, three per TMEM lane quarter over 16-column groups:
//               tcgen05.ld of P and Q, the cell test, codes, the
//               per-function min / max, the flag list
//   warps 14-21 converters: FP32 box -> three BF16 parts in the 128-byte
//               swizzled K-major layout (2-stage ring), and |x|^2 per row
// Every mbarrier wait is bounded (2 s): on expiry the kernel records
// GEEK_ERR_TIMEOUT, stops issuing, drains its own copies and MMAs, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int PT_M = 128;
constexpr int PT_BOX = 32;                         // FP32 columns per TMA box
constexpr int PT_F32_STAGES = 3;
constexpr int PT_F32_STAGE = PT_M * PT_BOX * 4;    // 16 KB
constexpr int PT_PART = PT_M * 128;                // one BF16 part of a 64-column k-block: 16 KB
constexpr int PT_SPLIT_STAGE = 3 * PT_PART;        // 48 KB
constexpr int PT_SPLIT_STAGES = 2;
constexpr int PT_NMAX = 128;                       // functions (padded) per launch
constexpr int PT_A_MAX = 3 * 96 * 2 * 128;         // image of A: 3 parts x N x nkb x 128 B (N * nkb <= 192)
constexpr int PT_CONV_WARPS = 8;
constexpr int PT_EPI_PER_Q = 3;                    // epilogue warps per TMEM lane quarter
constexpr int PT_EPI_WARPS = 4 * PT_EPI_PER_Q;
constexpr int PT_THREADS = 32 * (2 + PT_EPI_WARPS + PT_CONV_WARPS);
constexpr uint32_t PT_TMEM_COLS = 512;             // 2 buffers x (P, Q) x 128 columns
constexpr int PT_OFF_SPLIT = PT_A_MAX;
constexpr int PT_OFF_F32 = PT_OFF_SPLIT + PT_SPLIT_STAGES * PT_SPLIT_STAGE;
constexpr int PT_OFF_MISC = PT_OFF_F32 + PT_F32_STAGES * PT_F32_STAGE;
constexpr int PT_MISC = 6144;
constexpr int PT_SMEM = PT_OFF_MISC + PT_MISC + 1024;  // + alignment slack
static_assert(PT_SMEM <= 232448, "shared memory of one CTA");
static_assert(PT_A_MAX % 1024 == 0 && PT_OFF_F32 % 1024 == 0, "1 KB alignment of the swizzled tiles");

struct PtArgs {
    CUtensorMap tmX;            // x: {d, n} FP32, row pitch ldx * 4, box {32, 128}, no swizzle
    const uint8_t *aimg;        // [3][nkb][N rows][128 B] swizzled BF16 parts of A
    uint32_t aimg_bytes;
    const float *b, *anorm;     // F
    float inv_w;
    int srp;
    int64_t n;
    int d, F, N, nkb, nhalf;    // nhalf: 32-column boxes holding data (ceil(d / 32))
    float coef;                 // E = coef * |a_f| * |x|
    int32_t *codes;             // n x F
    int *fmin, *fmax;           // F
    uint64_t *flags;            // (global row << 16) | f
    unsigned long long *n_flags;
    int64_t flag_cap;
    int64_t row_base;
    int *err;
};

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

// byte offset of element (row r, column c in 0..63) in one swizzled part
__device__ __forceinline__ uint32_t sw128(int r, int c) {
    return (uint32_t)(((r >> 3) << 10) + ((r & 7) << 7) + ((((c >> 3) ^ (r & 7))) << 4) + ((c & 7) << 1));
}

// v = v1 + v2 + v3 (+ a residue below 2^-24 |v|), each a BF16
__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h1, __nv_bfloat16 &h2, __nv_bfloat16 &h3) {
    h1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h1);  // exact
    h2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h2);  // exact
    h3 = __float2bfloat16_rn(r2);
}

// the same split for two neighbouring columns, packed as BF16 pairs (the
// first column in the low half, as it sits at the lower address)
__device__ __forceinline__ void split3x2(float2 v, uint32_t &w1, uint32_t &w2, uint32_t &w3) {
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.x, v.y);
    const float2 f1 = __bfloat1622float2(h1);
    const float2 r1 = make_float2(v.x - f1.x, v.y - f1.y);  // exact
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(r1.x, r1.y);
    const float2 f2 = __bfloat1622float2(h2);
    const __nv_bfloat162 h3 = __floats2bfloat162_rn(r1.x - f2.x, r1.y - f2.y);  // differences exact
    w1 = *reinterpret_cast<const uint32_t *>(&h1);
    w2 = *reinterpret_cast<const uint32_t *>(&h2);
    w3 = *reinterpret_cast<const uint32_t *>(&h3);
}

// lane 0 waits; __syncwarp then orders the other lanes' reads after its
// acquire of the barrier phase
__device__ __forceinline__ bool wait_bcast(uint64_t *bar, uint32_t parity, int *err, int lane) {
    int ok = 0;
    if (lane == 0) ok = mbar_wait(bar, parity, err);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__global__ void __launch_bounds__(PT_THREADS, 1) k_project_tc(const __grid_constant__ PtArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sS = base + PT_OFF_SPLIT;
    uint8_t *sF = base + PT_OFF_F32;
    uint64_t *bars = (uint64_t *)(base + PT_OFF_MISC);
    uint64_t *a_full = bars;                        // 1
    uint64_t *f_full = bars + 1, *f_empty = bars + 4;    // 3 + 3
    uint64_t *s_full = bars + 7, *s_empty = bars + 9;    // 2 + 2
    uint64_t *acc_full = bars + 11, *acc_empty = bars + 13;
    uint64_t *nrm_full = bars + 15, *nrm_empty = bars + 17;
    uint64_t *done_bar = bars + 19;
    uint32_t *tmem_slot = (uint32_t *)(bars + 20);
    float *rownorm = (float *)(base + PT_OFF_MISC + 256);   // [2][128]
    int *s_min = (int *)(rownorm + 2 * PT_M);                // [128]
    int *s_max = s_min + PT_NMAX;                            // [128]
    float4 *s_pk = (float4 *)(s_max + PT_NMAX);              // [128] {b, alpha, beta, 0} of the cell test
    float *s_lim = (float *)(s_pk + PT_NMAX);                // max |a_f| / w, max |b_f| / w

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int i = 0; i < PT_F32_STAGES; i++) {
            mbar_init(&f_full[i], 1);
            mbar_init(&f_empty[i], PT_CONV_WARPS);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&s_full[i], PT_CONV_WARPS);
            mbar_init(&s_empty[i], 1);
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], PT_EPI_WARPS);
            mbar_init(&nrm_full[i], PT_CONV_WARPS);
            mbar_init(&nrm_empty[i], PT_EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int f = threadIdx.x; f < PT_NMAX; f += blockDim.x) {
        const float bb = f < A.F ? A.b[f] : 0.f, an = f < A.F ? A.anorm[f] : 0.f;
        s_min[f] = INT32_MAX;
        s_max[f] = INT32_MIN;
        // One FFMA bound of the cell test's window (fast loop of the epilogue),
        // Et = alpha |x| + beta >= the general loop's Et + 6e-8 for every p
        // the accumulator can hold (|p| <= |a_f| |x| + E): alpha and beta
        // carry 1e-5 for their own and the FFMA's FP32 rounding, the 6e-8
        // the rounding of tt - floor(tt) and of 1 - Et.
        float al, be;
        if (A.srp) {
            al = an * (A.coef * 1.000001f + 1.21e-7f) * 1.00001f;
            be = 1.1e-30f;
        } else {
            al = A.inv_w * an * (A.coef * 1.000001f + 5.02e-7f) * 1.00001f;
            be = A.inv_w * (fabsf(bb) * 5.02e-7f + 1.1e-30f) * 1.00001f + 6e-8f;
        }
        s_pk[f] = make_float4(bb, al, be, 0.f);
    }
    if (threadIdx.x == 0) {
        float am = 0.f, bm = 0.f;
        for (int f = 0; f < A.F; f++) {
            am = fmaxf(am, A.anorm[f]);
            bm = fmaxf(bm, fabsf(A.b[f]));
        }
        s_lim[0] = am * A.inv_w * 1.00001f;
        s_lim[1] = bm * A.inv_w * 1.00001f;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(PT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t ntiles = (A.n + PT_M - 1) / PT_M;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            mbar_expect_tx(a_full, A.aimg_bytes);
            bulk_load(su32(sA), A.aimg, A.aimg_bytes, a_full);
            uint64_t g = 0;
            uint32_t issued[PT_F32_STAGES] = {0, 0, 0};
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
                for (int hh = 0; hh < A.nhalf; hh++, g++) {
                    const int slot = (int)(g % PT_F32_STAGES);
                    const uint32_t u = (uint32_t)(g / PT_F32_STAGES);
                    if (!(ok = mbar_wait(&f_empty[slot], (u & 1) ^ 1, A.err))) break;
                    mbar_expect_tx(&f_full[slot], PT_F32_STAGE);
                    tma_load_2d(su32(sF + slot * PT_F32_STAGE), &A.tmX, hh * PT_BOX, (int)(t * PT_M), &f_full[slot]);
                    issued[slot] = u + 1;
                }
            // drain: every copy this thread issued has landed
            mbar_wait(a_full, 0, A.err, true);
            for (int s = 0; s < PT_F32_STAGES; s++)
                if (issued[s]) mbar_wait(&f_full[s], (issued[s] - 1) & 1, A.err, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = mbar_wait(a_full, 0, A.err);
            const uint32_t idesc = idesc_bf16(PT_M, A.N);
            const uint32_t abase = su32(sA);
            const uint32_t pstride = (uint32_t)A.nkb * A.N * 128;  // bytes between A's parts
            uint64_t s = 0;
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
                const int buf = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!(ok = mbar_wait(&acc_empty[buf], (ub & 1) ^ 1, A.err))) break;
                fence_after();
                const uint32_t dP = tmem + (uint32_t)(buf * 256), dQ = dP + 128;
                for (int kb = 0; kb < A.nkb && ok; kb++, s++) {
                    const int ss = (int)(s & 1);
                    const uint32_t us = (uint32_t)(s >> 1);
                    if (!(ok = mbar_wait(&s_full[ss], us & 1, A.err))) break;
                    fence_after();
                    const uint32_t x1 = su32(sS + ss * PT_SPLIT_STAGE), x2 = x1 + PT_PART, x3 = x2 + PT_PART;
                    const uint32_t a1 = abase + (uint32_t)kb * A.N * 128, a2 = a1 + pstride, a3 = a2 + pstride;
                    for (int ks = 0; ks < 4; ks++) {
                        if (kb * 64 + ks * 16 >= A.d) break;  // all-zero k-steps add nothing
                        const uint32_t o = ks * 32;
                        const uint32_t acc = (kb | ks) != 0;
                        mma_bf16(dP, sdesc(x1 + o), sdesc(a1 + o), idesc, acc);
                        mma_bf16(dQ, sdesc(x1 + o), sdesc(a2 + o), idesc, acc);
                        mma_bf16(dQ, sdesc(x2 + o), sdesc(a1 + o), idesc, 1);
                        mma_bf16(dQ, sdesc(x1 + o), sdesc(a3 + o), idesc, 1);
                        mma_bf16(dQ, sdesc(x2 + o), sdesc(a2 + o), idesc, 1);
                        mma_bf16(dQ, sdesc(x3 + o), sdesc(a1 + o), idesc, 1);
                    }
                    mma_commit(&s_empty[ss]);
                }
                if (ok) mma_commit(&acc_full[buf]);
            }
            // drain: all MMAs this thread issued have completed
            mma_commit(done_bar);
            mbar_wait(done_bar, 0, A.err, true);
        }
        __syncwarp();
    } else if (warp < 2 + PT_EPI_WARPS) {
        // ------------------------------------------------------ epilogue
        // PT_EPI_PER_Q warps share a TMEM lane quarter; warp e of a quarter
        // takes the 16-column groups e, e + PT_EPI_PER_Q, ...
        const int ew = warp - 2;
        const int q = warp & 3;  // TMEM lane quarter
        const int e = ew >> 2;   // column groups of this warp
        const int rloc = 32 * q + lane;
        const int ngrp = A.N / 16;
        bool ok = true;
        int64_t it = 0;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
            const int buf = (int)(it & 1);
            const uint32_t ub = (uint32_t)(it >> 1);
            if (!(ok = wait_bcast(&acc_full[buf], ub & 1, A.err, lane))) break;
            if (!(ok = wait_bcast(&nrm_full[buf], ub & 1, A.err, lane))) break;
            fence_after();
            const int64_t row = t * PT_M + rloc;
            const bool live = row < A.n;
            const float xn = sqrtf(rownorm[buf * PT_M + rloc]) * (1.f + 1e-4f);
            // |tt| <= (|a_f| |x| (1 + E) + |b_f|) / w stays far below 2^31 in every
            // row of the tile (E2LSH; SRP has no tt)
            const bool fastrows = __all_sync(0xffffffffu, live && (A.srp || s_lim[0] * xn + s_lim[1] < 1e9f));
            __syncwarp();
            if (lane == 0) mbar_arrive(&nrm_empty[buf]);
            for (int gi = e; gi < ngrp; gi += PT_EPI_PER_Q) {
                uint32_t rp[16], rq[16];
                const uint32_t tb = tmem + (uint32_t)(buf * 256 + gi * 16) + ((uint32_t)(32 * q) << 16);
                tmem_ld16_async(tb, rp);
                tmem_ld16_async(tb + 128, rq);
                tmem_wait_ld();
                uint32_t flagged = 0;
                int lmin = INT32_MAX, lmax = INT32_MIN;
                if (fastrows && gi * 16 + 16 <= A.F) {
                    // every row live, every column a function, no |tt| near 2^31:
                    // the cell test with the one-FFMA window, no guards
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float4 pk = s_pk[gi * 16 + j];
                        const float p = __uint_as_float(rp[j]) + __uint_as_float(rq[j]);
                        const float Et = fmaf(pk.y, xn, pk.z);
                        int code;
                        bool sure;
                        if (A.srp) {
                            code = p >= 0.f ? 1 : 0;
                            sure = fabsf(p) > Et;
                        } else {
                            const float tt = (p + pk.x) * A.inv_w;
                            const float c0 = floorf(tt);
                            const float fr = tt - c0;
                            code = (int)c0;
                            sure = fr >= Et && fr < 1.f - Et;
                        }
                        rp[j] = (uint32_t)code;
                        if (!sure) flagged |= 1u << j;
                        const int mn = __reduce_min_sync(0xffffffffu, code);
                        const int mx = __reduce_max_sync(0xffffffffu, code);
                        if (lane == j) {
                            lmin = mn;
                            lmax = mx;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int f = gi * 16 + j;
                        const bool fv = live && f < A.F;
                        const float4 pk = s_pk[f];
                        const float p = __uint_as_float(rp[j]) + __uint_as_float(rq[j]);
                        const float Et = fmaf(pk.y, xn, pk.z);
                        int code;
                        bool sure;
                        if (A.srp) {
                            code = p >= 0.f ? 1 : 0;
                            sure = fabsf(p) > Et;
                        } else {
                            const float tt = (p + pk.x) * A.inv_w;
                            const float c0 = floorf(tt);
                            const float fr = tt - c0;
                            const bool small = fabsf(tt) < 2.0e9f;
                            code = small ? (int)c0 : 0;
                            sure = small && fr >= Et && fr < 1.f - Et;
                        }
                        rp[j] = (uint32_t)code;  // the codes replace P in place
                        if (fv && !sure) flagged |= 1u << j;
                        const int mn = __reduce_min_sync(0xffffffffu, fv ? code : INT32_MAX);
                        const int mx = __reduce_max_sync(0xffffffffu, fv ? code : INT32_MIN);
                        if (lane == j) {
                            lmin = mn;
                            lmax = mx;
                        }
                    }
                }
                if (lane < 16 && gi * 16 + lane < A.F && lmin <= lmax) {
                    atomicMin(&s_min[gi * 16 + lane], lmin);
                    atomicMax(&s_max[gi * 16 + lane], lmax);
                }
                if (live) {
                    int32_t *dst = A.codes + row * A.F + gi * 16;
                    const int cnt = min(16, A.F - gi * 16);
                    if (cnt == 16 && (A.F & 3) == 0) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<int4 *>(dst + j) =
                                make_int4((int)rp[j], (int)rp[j + 1], (int)rp[j + 2], (int)rp[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (j < cnt) dst[j] = (int)rp[j];
                    }
                }
                // flag list: one atomic per warp and group
                const unsigned nf = __popc(flagged);
                unsigned incl = nf;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
                if (tot) {
                    unsigned long long pos = 0;
                    if (lane == 31) pos = atomicAdd(A.n_flags, (unsigned long long)tot);
                    pos = __shfl_sync(0xffffffffu, pos, 31) + (incl - nf);
                    while (flagged) {
                        const int j = __ffs(flagged) - 1;
                        flagged &= flagged - 1;
                        if ((int64_t)pos < A.flag_cap)
                            A.flags[pos] = ((uint64_t)(A.row_base + row) << 16) | (uint64_t)(gi * 16 + j);
                        pos++;
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    } else {
        // ------------------------------------------------------ converters
        const int cw = warp - 2 - PT_EPI_WARPS;
        const int c0 = 2 * (lane & 15);
        bool ok = true;
        uint64_t g = 0, s = 0;
        int64_t it = 0;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
            float xs[8];
#pragma unroll
            for (int i = 0; i < 8; i++) xs[i] = 0.f;
            for (int hh = 0; hh < A.nhalf && ok; hh++, g++) {
                const int kb = hh >> 1, h = hh & 1;
                const int ss = (int)(s & 1);
                if (h == 0 && !(ok = wait_bcast(&s_empty[ss], ((uint32_t)(s >> 1) & 1) ^ 1, A.err, lane))) break;
                const int fs = (int)(g % PT_F32_STAGES);
                if (!(ok = wait_bcast(&f_full[fs], (uint32_t)(g / PT_F32_STAGES) & 1, A.err, lane))) break;
                const float *src = reinterpret_cast<const float *>(sF + fs * PT_F32_STAGE);
                uint8_t *dst = sS + ss * PT_SPLIT_STAGE;
                const int kc = h * 32 + c0;  // column inside the k-block
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    // lanes 16-31 take the row four below: the two half-warps
                    // then write disjoint bank groups of the swizzled rows
                    const int r = cw * 16 + (i & 3) + ((i >> 2) << 3) + ((lane >> 4) << 2);
                    const float2 v = *reinterpret_cast<const float2 *>(src + r * PT_BOX + c0);
                    xs[i] = fmaf(v.x, v.x, fmaf(v.y, v.y, xs[i]));
                    uint32_t w1, w2, w3;
                    split3x2(v, w1, w2, w3);
                    const uint32_t o = sw128(r, kc);
                    *reinterpret_cast<uint32_t *>(dst + o) = w1;
                    *reinterpret_cast<uint32_t *>(dst + PT_PART + o) = w2;
                    *reinterpret_cast<uint32_t *>(dst + 2 * PT_PART + o) = w3;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&f_empty[fs]);
                if (h == 1 || hh == A.nhalf - 1) {
                    // this k-block is complete: hand it to the tensor core
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&s_full[ss]);
                    s++;
                }
            }
            if (!ok) break;
            // |x|^2 of the warp's 16 rows: lanes 0 and 16 end with the sums
#pragma unroll
            for (int i = 0; i < 8; i++) {
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) xs[i] += __shfl_xor_sync(0xffffffffu, xs[i], o);
            }
            const int buf = (int)(it & 1);
            if (!(ok = wait_bcast(&nrm_empty[buf], ((uint32_t)(it >> 1) & 1) ^ 1, A.err, lane))) break;
            if ((lane & 15) == 0) {
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int r = cw * 16 + (i & 3) + ((i >> 2) << 3) + ((lane >> 4) << 2);
                    rownorm[buf * PT_M + r] = xs[i];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&nrm_full[buf]);
        }
    }
    fence_before();
    __syncthreads();
    for (int f = threadIdx.x; f < A.F; f += blockDim.x)
        if (s_min[f] <= s_max[f]) {
            atomicMin(&A.fmin[f], s_min[f]);
            atomicMax(&A.fmax[f], s_max[f]);
        }
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PT_TMEM_COLS) : "memory");
    }
}

// The swizzled image of A's three BF16 parts, [part][k-block][N rows][64
// columns], zero beyond F rows and d columns; thread per (row, column).
__global__ void k_pt_aimg(const float *__restrict__ a, int F, int d, int N, int nkb, uint8_t *__restrict__ img) {
    const int total = N * nkb * 64;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int f = e / (nkb * 64), kc = e % (nkb * 64);
        const int kb = kc >> 6, c = kc & 63;
        const float v = (f < F && kc < d) ? a[(int64_t)f * d + kc] : 0.f;
        __nv_bfloat16 h1, h2, h3;
        split3(v, h1, h2, h3);
        const size_t pstride = (size_t)nkb * N * 128;
        const size_t o = (size_t)kb * N * 128 + sw128(f, c);
        *reinterpret_cast<__nv_bfloat16 *>(img + o) = h1;
        *reinterpret_cast<__nv_bfloat16 *>(img + pstride + o) = h2;
        *reinterpret_cast<__nv_bfloat16 *>(img + 2 * pstride + o) = h3;
    }
}

}  // namespace

bool proj_tc_eligible(const float *x, int64_t ldx, int d, int F) {
    const int N = (F + 31) / 32 * 32;
    const int nkb = (d + 63) / 64;
    return d >= 1 && d <= 128 && F >= 1 && N <= PT_NMAX && N * nkb <= 192 && (ldx & 3) == 0 &&
           ((uintptr_t)x & 15) == 0;
}

// Window coefficient of the split tensor-core projection (see the header).
static float proj_tc_coef(int d) {
    const double nk = (double)((d + 15) / 16);
    const double u20 = 9.5367431640625e-07;  // 2^-20
    const double c = nk * u20 * 1.0079 + 5.0 * nk * u20 * 0.0079 + 5.9604644775390625e-08 * 1.01 +
                     2.384185791015625e-07 * 1.01 + (double)d * 1.12e-16;
    return (float)(1.01 * c);
}

geek_status proj_tc_launch(geek_ctx *ctx, Scratch &scr, const ProjArgs &P, int *err, cudaStream_t st) {
    const int F = P.F, d = P.d;
    const int N = (F + 31) / 32 * 32;
    const int nkb = (d + 63) / 64;
    PtArgs A;
    memset(&A, 0, sizeof A);
    // a layout the tensor map cannot describe: the caller takes the FP32 path
    if (encode_2d(ctx, &A.tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)P.x, (uint64_t)d, (uint64_t)P.n,
                  (uint64_t)P.ldx * 4, PT_BOX, PT_M, CU_TENSOR_MAP_SWIZZLE_NONE) != GEEK_OK)
        return GEEK_ERR_UNSUPPORTED;
    const size_t img_bytes = (size_t)3 * nkb * N * 128;
    uint8_t *img;
    GK_TRY(scr.alloc(&img, img_bytes));
    GK_COUNT();
    k_pt_aimg<<<(N * nkb * 64 + 255) / 256, 256, 0, st>>>(P.a, F, d, N, nkb, img);
    GK_LAUNCH(ctx);
    A.aimg = img;
    A.aimg_bytes = (uint32_t)img_bytes;
    A.b = P.b;
    A.anorm = P.anorm;
    A.inv_w = P.inv_w;
    A.srp = P.srp;
    A.n = P.n;
    A.d = d;
    A.F = F;
    A.N = N;
    A.nkb = nkb;
    A.nhalf = (d + PT_BOX - 1) / PT_BOX;
    A.coef = proj_tc_coef(d);
    A.codes = P.codes;
    A.fmin = P.fmin;
    A.fmax = P.fmax;
    A.flags = P.flags;
    A.n_flags = P.n_flags;
    A.flag_cap = P.flag_cap;
    A.row_base = P.row_base;
    A.err = err;
    static bool attr_done = false;
    if (!attr_done) {
        GK_CUDA(ctx, cudaFuncSetAttribute(k_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM));
        attr_done = true;
    }
    const int64_t ntiles = ceil_div(P.n, PT_M);
    const int grid = (int)std::min<int64_t>(ntiles, ctx->num_sms);
    GK_COUNT();
    k_project_tc<<<grid, PT_THREADS, PT_SMEM, st>>>(A);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}
