// Data transformation kernels (Sect. 3.1): dense E2LSH / sign projections
// with an FP64 boundary recheck, MinHash of sets and of categorical tokens
// (Eq. 2), and the order-preserving packing of each table's K-tuple into a
// 64/128-bit sort key.
#include "common.cuh"
#include "internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// FP32 SIMT projection P = X A^T with the E2LSH / SRP epilogue.
//
// Rigorous window.  For one element, v = a.x is the exact real dot product,
// p its FP32 value accumulated with FMA in any order, s64 the FP64 reference
// (products exact, sequential sum).  |p - v| <= gamma_d * sum|a_j x_j| and
// |s64 - v| <= d 2^-53 sum|a_j x_j|, and sum|a_j x_j| <= |a| |x| (Cauchy-
// Schwarz), so s64 lies within E = (gamma_d + d 2^-53) |a| |x| of p.  The
// reference code s -> floor(rn(rn(s + b) / w)) is monotone in s, so when the
// whole interval maps into one integer cell the code is certain; otherwise
// the element goes to the FP64 recheck list.  The cell test itself runs in
// FP32 with its own rounding terms added to the window.
// ---------------------------------------------------------------------------
constexpr int PJ_KC = 32;       // d-chunk staged in shared memory
constexpr int PJ_FPT = 8;       // functions per thread
constexpr int PJ_RPT = 8;       // rows per thread
constexpr int PJ_MAXT = 256;    // threads per block (upper bound)



// One block: rows [tile * TR, tile * TR + TR) of one instance.  BATCH = false:
// A describes the only instance (read from the parameter space, which the
// inner loops use as operands directly).  BATCH = true: block b belongs to
// instance i with tile_off[i] <= b < tile_off[i + 1], whose pointers and
// sizes P[i] replace A's; the thread layout (F, FPAD, FG, RG) and the flag
// list are common to the batch and stay A's.
template <bool BATCH>
__global__ void __launch_bounds__(PJ_MAXT, 2) k_project_fp32(ProjArgs A, const ProjArgs *__restrict__ P,
                                                          const int64_t *__restrict__ tile_off, int count) {
    int64_t tile = blockIdx.x;
    if (BATCH) {
        __shared__ int s_i;
        if (threadIdx.x == 0) s_i = find_inst(tile_off, count, blockIdx.x);
        __syncthreads();
        const ProjArgs &Q = P[s_i];
        tile = (int64_t)blockIdx.x - tile_off[s_i];
        A.x = Q.x;
        A.ldx = Q.ldx;
        A.n = Q.n;
        A.d = Q.d;
        A.a = Q.a;
        A.b = Q.b;
        A.anorm = Q.anorm;
        A.w = Q.w;
        A.inv_w = Q.inv_w;
        A.codes = Q.codes;
        A.fmin = Q.fmin;
        A.fmax = Q.fmax;
        A.row_base = Q.row_base;
    }
    extern __shared__ float sm[];
    const int TR = A.RG * PJ_RPT;
    // Two stages of row-major chunks, 32 k-values (128 B) per row: xs [TR][32]
    // and as [FPAD][32].  The 16-byte piece j of row r sits at position
    // j ^ ((r >> 3) & 7), so the float4 reads of a quarter warp (rows 8
    // apart) fall in different banks.  With 16-byte aligned rows the stages
    // are filled by cp.async one chunk ahead of the arithmetic.
    const int SR = TR + A.FPAD;  // rows per stage
    float *st0 = sm, *st1 = sm + (size_t)SR * PJ_KC;
    __shared__ int smin[512], smax[512];  // F <= 512 checked on the host
    const int t = threadIdx.x;
    const int nthr = A.FG * A.RG;
    const int fg = t % A.FG, rg = t / A.FG;
    const bool active = t < nthr;
    const int64_t row0 = tile * TR;
    for (int f = t; f < A.F; f += blockDim.x) {
        smin[f] = INT32_MAX;
        smax[f] = INT32_MIN;
    }
    float acc[PJ_RPT][PJ_FPT];
    float xsq[PJ_RPT];
#pragma unroll
    for (int r = 0; r < PJ_RPT; r++) {
        xsq[r] = 0.f;
#pragma unroll
        for (int c = 0; c < PJ_FPT; c++) acc[r][c] = 0.f;
    }
    const bool vec = ((A.ldx & 3) == 0) && ((A.d & 3) == 0) && (((uintptr_t)A.x & 15) == 0) &&
                     (((uintptr_t)A.a & 15) == 0);
    // fills stage `buf` with the chunk at k0: rows 0..TR-1 from X, then FPAD
    // rows from A (zeros outside the data)
    auto stage = [&](float *buf, int k0) {
        for (int e = t; e < SR * 8; e += blockDim.x) {
            const int r = e >> 3, j = e & 7;
            const int k = k0 + 4 * j;
            const float *src = nullptr;
            bool in = false;
            int sw;  // row index within its own matrix (the swizzle key)
            if (r < TR) {
                const int64_t row = row0 + r;
                in = row < A.n;
                src = A.x + row * A.ldx + k;
                sw = r;
            } else {
                const int f = r - TR;
                in = f < A.F;
                src = A.a + (int64_t)f * A.d + k;
                sw = f;
            }
            float *dst = buf + r * PJ_KC + 4 * (j ^ ((sw >> 3) & 7));
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
    const int nchunks = (A.d + PJ_KC - 1) / PJ_KC;
    stage(st0, 0);
    for (int ci = 0; ci < nchunks; ci++) {
        float *cur = (ci & 1) ? st1 : st0;
        if (ci + 1 < nchunks) {
            stage((ci & 1) ? st0 : st1, (ci + 1) * PJ_KC);
            if (vec) asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else if (vec) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (active) {
            const float *xb = cur, *ab = cur + (size_t)TR * PJ_KC;
            const int kmax = min(PJ_KC, A.d - ci * PJ_KC);
            for (int jb = 0; jb < (kmax + 3) / 4; jb++) {
                float4 xv[PJ_RPT];
#pragma unroll
                for (int q = 0; q < PJ_RPT; q++) {
                    const int r = rg * PJ_RPT + q;
                    xv[q] = *reinterpret_cast<const float4 *>(xb + r * PJ_KC + 4 * (jb ^ ((r >> 3) & 7)));
                    xsq[q] = fmaf(xv[q].x, xv[q].x, fmaf(xv[q].y, xv[q].y, fmaf(xv[q].z, xv[q].z, fmaf(xv[q].w, xv[q].w, xsq[q]))));
                }
#pragma unroll
                for (int c = 0; c < PJ_FPT; c++) {
                    const int f = fg * PJ_FPT + c;
                    const float4 av = *reinterpret_cast<const float4 *>(ab + f * PJ_KC + 4 * (jb ^ ((f >> 3) & 7)));
#pragma unroll
                    for (int q = 0; q < PJ_RPT; q++) {
                        acc[q][c] = fmaf(xv[q].x, av.x, acc[q][c]);
                        acc[q][c] = fmaf(xv[q].y, av.y, acc[q][c]);
                        acc[q][c] = fmaf(xv[q].z, av.z, acc[q][c]);
                        acc[q][c] = fmaf(xv[q].w, av.w, acc[q][c]);
                    }
                }
            }
        }
        __syncthreads();  // the next stage() overwrites this buffer
    }
    __syncthreads();
    unsigned nfl = 0;
    uint64_t flagmask = 0;  // bit r*8 + c: element (row r, function c) is uncertain
    if (active) {
        const float gam = (float)A.d * 6.0e-8f;  // >= gamma_d(fp32) + d 2^-53, norms' own error
        int lmin[PJ_FPT], lmax[PJ_FPT];
#pragma unroll
        for (int c = 0; c < PJ_FPT; c++) {
            lmin[c] = INT32_MAX;
            lmax[c] = INT32_MIN;
        }
#pragma unroll
        for (int r = 0; r < PJ_RPT; r++) {
            const int64_t row = row0 + rg * PJ_RPT + r;
            if (row >= A.n) continue;
            const float xn = sqrtf(xsq[r]) * 1.0001f;
            int32_t out[PJ_FPT];
#pragma unroll
            for (int c = 0; c < PJ_FPT; c++) {
                const int f = fg * PJ_FPT + c;
                out[c] = 0;
                if (f >= A.F) continue;
                const float p = acc[r][c];
                const float E = gam * A.anorm[f] * xn + 1e-30f;
                int code;
                bool sure;
                if (A.srp) {
                    // s64 in [p - E, p + E]; FP32 subtraction slack 2^-23 |p|
                    const float Es = E + fabsf(p) * 1.2e-7f;
                    code = p >= 0.f ? 1 : 0;
                    sure = (p - Es > 0.f) || (p + Es < 0.f);
                } else {
                    const float bb = A.b[f];
                    const float tt = (p + bb) * A.inv_w;
                    // window in t-space: model error E/w plus rounding of
                    // p + b, of * (1/w) and of the comparisons (4 ulps)
                    const float Et = (E + (fabsf(p) + fabsf(bb) + E) * 2.5e-7f) * A.inv_w + fabsf(tt) * 2.5e-7f;
                    const float c0 = floorf(tt);
                    code = fabsf(tt) < 2.0e9f ? (int)c0 : 0;
                    sure = (tt - Et >= c0) && (tt + Et < c0 + 1.f) && fabsf(tt) < 2.0e9f;
                }
                out[c] = code;
                if (!sure) flagmask |= 1ull << (r * PJ_FPT + c);
                lmin[c] = min(lmin[c], code);
                lmax[c] = max(lmax[c], code);
            }
            int32_t *dst = A.codes + row * A.F + fg * PJ_FPT;
            if (fg * PJ_FPT + PJ_FPT <= A.F && (A.F % 4) == 0) {
                reinterpret_cast<int4 *>(dst)[0] = make_int4(out[0], out[1], out[2], out[3]);
                reinterpret_cast<int4 *>(dst)[1] = make_int4(out[4], out[5], out[6], out[7]);
            } else {
                for (int c = 0; c < PJ_FPT; c++)
                    if (fg * PJ_FPT + c < A.F) dst[c] = out[c];
            }
        }
#pragma unroll
        for (int c = 0; c < PJ_FPT; c++) {
            const int f = fg * PJ_FPT + c;
            if (f < A.F && lmin[c] <= lmax[c]) {
                atomicMin(&smin[f], lmin[c]);
                atomicMax(&smax[f], lmax[c]);
            }
        }
        nfl = __popcll(flagmask);
    }
    // one global atomic per block for the flag list
    __shared__ unsigned s_tot;
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_wsum[PJ_MAXT / 32];
    {
        const int lane = t & 31, warp = t >> 5;
        unsigned x = nfl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        if (t == 0) {
            unsigned run = 0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) {
                unsigned v = s_wsum[w];
                s_wsum[w] = run;
                run += v;
            }
            s_tot = run;
            s_base = run ? atomicAdd(A.n_flags, (unsigned long long)run) : 0ull;
        }
        __syncthreads();
        unsigned long long pos = s_base + s_wsum[warp] + x - nfl;
        while (flagmask) {
            const int bit = __ffsll(flagmask) - 1;
            flagmask &= flagmask - 1;
            const int64_t row = row0 + rg * PJ_RPT + bit / PJ_FPT;
            const int f = fg * PJ_FPT + bit % PJ_FPT;
            if ((int64_t)pos < A.flag_cap) A.flags[pos] = ((uint64_t)(A.row_base + row) << 16) | (uint64_t)f;
            pos++;
        }
    }
    __syncthreads();
    for (int f = t; f < A.F; f += blockDim.x) {
        if (smin[f] != INT32_MAX) {
            atomicMin(&A.fmin[f], smin[f]);
            atomicMax(&A.fmax[f], smax[f]);
        }
    }
}


__global__ void k_row_norms(const float *__restrict__ a, int F, int d, float *__restrict__ out) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    float s = 0.f;
    for (int j = 0; j < d; j++) s = fmaf(a[(int64_t)f * d + j], a[(int64_t)f * d + j], s);
    out[f] = sqrtf(s) * 1.0001f;
}

// Second stage for flagged elements: the dot product again in compensated
// FP32 (TwoProduct by FMA, TwoSum, error terms summed separately, after Ogita,
// Rump and Oishi's Dot2).  With the FP64 reference's own error this gives an
// interval of width ~1e-6 |a||x| around s64; if the monotone reference map
// sends both ends to one code the element is settled here, otherwise it goes
// on to the FP64 list (about one element in 10^7 at d = 128).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Eight lanes take one flagged element: lane s runs Dot2 over its
// coordinates 4s..4s+3, 4s+32.. (in order), TwoProduct p + h = a_j x_j,
// TwoSum sh + er = sh + p, error terms er + h summed in sc; the eight
// (sh, sc) pairs then merge in a tree of TwoSums (sh + sh', the new error
// added to sc + sc').  Every TwoSum and TwoProduct is error-free, so sh + the
// exact sum of all error terms is the exact dot product, and sc carries
// those 2d - 1 terms summed in floating point; each product's partial sums
// pass through at most d - 1 non-trivial TwoSums, as in the sequential
// order, so Ogita, Rump and Oishi's bound for Dot2 still holds: |sh + sc -
// a.x| <= u |a.x| + gamma_d^2 sum|a_j x_j| <= 2.2 (2d)(d+1) u^2 |a||x| beyond
// the final rounding.  A warp takes 32 flags: in step r its four lane groups
// take flags 4r .. 4r+3, and the result of flag m goes to lane m, which
// then makes the decision for its own flag (the FP64 part runs with 32
// flags per warp instruction).  The groups' loads of a row are 128 bytes
// apiece, where a thread per flag spread a warp's loads over 32 rows.
// Flag entries carry global rows (row_base + local row); instance i holds
// global rows [row_off[i], row_off[i + 1]).
__global__ void __launch_bounds__(256) k_recheck_dot2(
    const ProjArgs *__restrict__ P, const int64_t *__restrict__ row_off, int count, int srp, int F,
    const uint64_t *__restrict__ flags, const unsigned long long *__restrict__ n_flags, int64_t cap,
    uint64_t *__restrict__ flags2, unsigned long long *__restrict__ n_flags2) {
    const int64_t nf = min((int64_t)*n_flags, cap);
    const double u = 5.9604644775390625e-08;  // 2^-24
    const int lane = threadIdx.x & 31, grp = lane >> 3, sub = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q0 = warp * 32; q0 < nf; q0 += nwarps * 32) {
        float msh = 0.f, msc = 0.f, mxx = 0.f;  // this lane's own flag q0 + lane
        for (int r = 0; r < 8; r++) {
            const int64_t q = q0 + 4 * r + grp;
            float sh = 0.f, sc = 0.f, xx = 0.f;
            if (q < nf) {
                const uint64_t e = flags[q];
                const ProjArgs &A = P[find_inst(row_off, count, (int64_t)(e >> 16))];
                const int d = A.d;
                const float *xr = A.x + ((int64_t)(e >> 16) - A.row_base) * A.ldx;
                const float *ar = A.a + (int64_t)(e & 0xFFFF) * d;
                auto term = [&](float av, float xv) {
                    const float p = __fmul_rn(av, xv);
                    const float h = fmaf(av, xv, -p);  // exact product error
                    float t, er;
                    two_sum(sh, p, t, er);
                    sh = t;
                    sc = __fadd_rn(sc, __fadd_rn(er, h));
                    xx = fmaf(xv, xv, xx);
                };
                if (((d & 3) == 0) && ((((uintptr_t)xr) | ((uintptr_t)ar)) & 15) == 0) {
                    for (int j = 4 * sub; j < d; j += 32) {
                        const float4 av = *reinterpret_cast<const float4 *>(ar + j);
                        const float4 xv = *reinterpret_cast<const float4 *>(xr + j);
                        term(av.x, xv.x);
                        term(av.y, xv.y);
                        term(av.z, xv.z);
                        term(av.w, xv.w);
                    }
                } else {
                    for (int b = 4 * sub; b < d; b += 32)
                        for (int j = b; j < min(b + 4, d); j++) term(ar[j], xr[j]);
                }
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float sh2 = __shfl_xor_sync(0xffffffffu, sh, o);
                const float sc2 = __shfl_xor_sync(0xffffffffu, sc, o);
                const float xx2 = __shfl_xor_sync(0xffffffffu, xx, o);
                float t, er;
                two_sum(sh, sh2, t, er);
                sh = t;
                sc = __fadd_rn(__fadd_rn(sc, sc2), er);
                xx = __fadd_rn(xx, xx2);
            }
            // flag 4r + g (group g) belongs to lane 4r + g
            const int src = (lane & 3) << 3;
            const float vsh = __shfl_sync(0xffffffffu, sh, src);
            const float vsc = __shfl_sync(0xffffffffu, sc, src);
            const float vxx = __shfl_sync(0xffffffffu, xx, src);
            if ((lane >> 2) == r) {
                msh = vsh;
                msc = vsc;
                mxx = vxx;
            }
        }
        const int64_t q = q0 + lane;
        if (q >= nf) continue;
        const uint64_t e = flags[q];
        const ProjArgs &A = P[find_inst(row_off, count, (int64_t)(e >> 16))];
        const int d = A.d;
        const int64_t row = (int64_t)(e >> 16) - A.row_base;
        const int f = (int)(e & 0xFFFF);
        const double w = A.wd;
        const double cfac = 2.2 * (2.0 * d) * (d + 1.0) * u * u + (double)d * 2.220446049250313e-16;
        const double S = (double)msh + (double)msc;
        const double an = (double)A.anorm[f], xn = (double)(sqrtf(mxx) * (1.0f + 1.0e-3f));
        const double E = cfac * an * xn + fabs(S) * 8.881784197001252e-16 + (double)d * 1e-40 + 1e-300;
        const double lo = S - E, hi = S + E;
        bool sure;
        int code;
        if (srp) {
            sure = lo >= 0.0 || hi < 0.0;
            code = lo >= 0.0 ? 1 : 0;
        } else {
            const double bb = (double)A.b[f];
            const double tl = floor(__ddiv_rn(__dadd_rn(lo, bb), w));
            const double th = floor(__ddiv_rn(__dadd_rn(hi, bb), w));
            sure = tl == th && tl >= -2147483648.0 && tl <= 2147483647.0;
            code = sure ? (int)tl : 0;
        }
        if (sure) {
            A.codes[row * F + f] = code;
            // the bounds only move outwards: a code inside a value read
            // earlier is inside the final one, and needs no atomic
            if (code < *(volatile int *)&A.fmin[f]) atomicMin(&A.fmin[f], code);
            if (code > *(volatile int *)&A.fmax[f]) atomicMax(&A.fmax[f], code);
        } else {
            const unsigned long long slot = atomicAdd(n_flags2, 1ull);
            flags2[slot] = e;  // slot < nf <= cap
        }
    }
}

// FP64 recheck of flagged elements with the reference sequence: products of
// the float inputs (exact in FP64), summed in j order, then (s + b) / w,
// each step rounded to nearest; no fused multiply-add.
__global__ void k_recheck_fp64(const ProjArgs *__restrict__ P, const int64_t *__restrict__ row_off, int count,
                               int srp, int F, const uint64_t *__restrict__ flags,
                               const unsigned long long *__restrict__ n_flags, int64_t cap,
                               int *__restrict__ status) {
    const int64_t nf = min((int64_t)*n_flags, cap);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nf;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = flags[q];
        const ProjArgs &A = P[find_inst(row_off, count, (int64_t)(e >> 16))];
        const int d = A.d;
        const int64_t row = (int64_t)(e >> 16) - A.row_base;
        const int f = (int)(e & 0xFFFF);
        const float *xr = A.x + row * A.ldx;
        const float *ar = A.a + (int64_t)f * d;
        double s = 0.0;
        for (int j = 0; j < d; j++) s = __dadd_rn(s, __dmul_rn((double)ar[j], (double)xr[j]));
        int code;
        if (srp) {
            code = s >= 0.0 ? 1 : 0;
        } else {
            const double t = __ddiv_rn(__dadd_rn(s, (double)A.b[f]), A.wd);
            const double fl = floor(t);
            if (!(fl >= -2147483648.0 && fl <= 2147483647.0)) {
                atomicExch(status, (int)GEEK_ERR_OVERFLOW);
                continue;
            }
            code = (int)fl;
        }
        A.codes[row * F + f] = code;
        atomicMin(&A.fmin[f], code);
        atomicMax(&A.fmax[f], code);
    }
}

// ---------------------------------------------------------------------------
// MinHash (Eq. 2): warp per set, lane over functions, items broadcast by
// shuffles; every lane keeps FPL running minima.
// ---------------------------------------------------------------------------
// hash of one token: 32-bit items, or the 64-bit tokens of a DOPH reduction
// (the same family, h = ((A x + B) mod 2^64) >> 32, over the whole token)
__device__ __forceinline__ uint32_t mh_token(uint64_t A, uint64_t B, uint32_t x) { return mh_hash32(A, B, x); }
__device__ __forceinline__ uint32_t mh_token(uint64_t A, uint64_t B, uint64_t x) {
    return (uint32_t)((A * x + B) >> 32);
}

template <int FPL, bool FIXED, typename TOK = uint32_t>
__global__ void __launch_bounds__(256) k_minhash(int64_t n, const int64_t *__restrict__ off,
                                                 int row_len, const TOK *__restrict__ items,
                                                 int F, const uint64_t *__restrict__ A,
                                                 const uint64_t *__restrict__ B,
                                                 uint32_t *__restrict__ out, int out_ld) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t ca[FPL], cb[FPL];
#pragma unroll
    for (int q = 0; q < FPL; q++) {
        int f = lane + 32 * q;
        ca[q] = f < F ? A[f] : 0;
        cb[q] = f < F ? B[f] : 0;
    }
    for (int64_t i = warp; i < n; i += nwarps) {
        int64_t s, e;
        if (FIXED) {
            s = i * row_len;
            e = s + row_len;
        } else {
            s = off[i];
            e = off[i + 1];
        }
        uint32_t m[FPL];
#pragma unroll
        for (int q = 0; q < FPL; q++) m[q] = 0xFFFFFFFFu;
        for (int64_t base = s; base < e; base += 32) {
            const int cnt = (int)min((int64_t)32, e - base);
            const TOK mine = lane < cnt ? items[base + lane] : (TOK)0;
            for (int j = 0; j < cnt; j++) {
                const TOK v = __shfl_sync(0xffffffffu, mine, j);
#pragma unroll
                for (int q = 0; q < FPL; q++) m[q] = min(m[q], mh_token(ca[q], cb[q], v));
            }
        }
#pragma unroll
        for (int q = 0; q < FPL; q++) {
            int f = lane + 32 * q;
            if (f < F) out[i * out_ld + f] = m[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Key layout and packing.
// ---------------------------------------------------------------------------
// One block per instance (blockIdx.x; its F = L*K1 functions and L tables
// at offsets blockIdx.x * F and blockIdx.x * L): per function bit width of
// (max - min); per table total; status.
__global__ void k_key_layout(const int *__restrict__ fmin, const int *__restrict__ fmax, int L,
                             int K1, int K2, int *__restrict__ bits, int *__restrict__ tbits,
                             int *__restrict__ status) {
    fmin += (int64_t)blockIdx.x * L * K1;
    fmax += (int64_t)blockIdx.x * L * K1;
    bits += (int64_t)blockIdx.x * L * K1;
    tbits += (int64_t)blockIdx.x * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int tot = 0;
        for (int k = 0; k < K1; k++) {
            int f = l * K1 + k;
            uint32_t range = fmin[f] <= fmax[f] ? (uint32_t)((int64_t)fmax[f] - (int64_t)fmin[f]) : 0u;
            int bl = 32 - __clz(range);
            bits[f] = bl;
            tot += bl;
        }
        tot += 32 * K2;
        tbits[l] = tot;
        if (tot > 128) atomicExch(status, (int)GEEK_ERR_OVERFLOW);
    }
}

__device__ __forceinline__ void shl_or(uint64_t &hi, uint64_t &lo, int b, uint64_t v) {
    if (b == 0) return;
    hi = (hi << b) | (lo >> (64 - b));
    lo = (lo << b) | v;
}

// key of table l for object i: fields codes[l*K1+k] - min (bits[f] wide),
// then K2 MinHash values (32 bits each), the first field most significant.
// One thread per object walks all L tables, so each code row is read once;
// a block first copies its objects' code rows to shared memory with
// coalesced loads (row stride F1 | 1 words: conflict-free row reads), when
// they fit (PK_STAGE_MAX codes per row).
constexpr int PK_THREADS = 256, PK_STAGE_MAX = 128;

// copies `rows` consecutive code rows (F1 codes each, from row r0) to shared
// rows of stride F1 | 1; the (row, column) of element e advance by fixed
// steps instead of a division per element
__device__ __forceinline__ void pk_stage_rows(int32_t *cs, const int32_t *__restrict__ codes, int64_t r0, int rows,
                                              int F1) {
    const int rs = F1 | 1;
    const int32_t *src = codes + r0 * F1;
    const int total = rows * F1;
    if ((F1 & 3) == 0 && ((uintptr_t)src & 15) == 0) {
        // 16-byte loads, four in flight per thread: a row holds a whole
        // number of them, so each vector's (row, column) comes from one
        // division
        const int nv = total >> 2, fv = F1 >> 2;
        for (int v0 = threadIdx.x; v0 < nv; v0 += 4 * PK_THREADS) {
            int4 q[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int v = v0 + u * PK_THREADS;
                q[u] = v < nv ? reinterpret_cast<const int4 *>(src)[v] : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int v = v0 + u * PK_THREADS;
                if (v >= nv) break;
                const int r = v / fv, c = (v - r * fv) * 4;
                int32_t *d = cs + r * rs + c;
                d[0] = q[u].x;
                d[1] = q[u].y;
                d[2] = q[u].z;
                d[3] = q[u].w;
            }
        }
        return;
    }
    const int dr = PK_THREADS / F1, dc = PK_THREADS % F1;
    int r = threadIdx.x / F1, c = threadIdx.x % F1;
    for (int e = threadIdx.x; e < total; e += PK_THREADS) {
        cs[r * rs + c] = src[e];
        r += dr;
        c += dc;
        if (c >= F1) {
            c -= F1;
            r++;
        }
    }
}
__global__ void __launch_bounds__(PK_THREADS) k_pack_keys(int64_t n, int L, const int32_t *__restrict__ codes,
                                                          int F1, int K1, const int *__restrict__ fmin,
                                                          const int *__restrict__ bits,
                                                          const uint32_t *__restrict__ mh, int F2, int K2,
                                                          uint64_t *__restrict__ klo, uint64_t *__restrict__ khi) {
    extern __shared__ int32_t cs[];
    __shared__ int s_min[PK_STAGE_MAX], s_bits[PK_STAGE_MAX];
    const bool staged = F1 > 0 && F1 <= PK_STAGE_MAX;
    const int rs = F1 | 1;
    if (staged) {
        for (int f = threadIdx.x; f < F1; f += PK_THREADS) {
            s_min[f] = fmin[f];
            s_bits[f] = bits[f];
        }
    }
    const int *fm = staged ? s_min : fmin;
    const int *bt = staged ? s_bits : bits;
    for (int64_t i0 = (int64_t)blockIdx.x * PK_THREADS; i0 < n; i0 += (int64_t)gridDim.x * PK_THREADS) {
        const int64_t i = i0 + threadIdx.x;
        if (staged) {
            __syncthreads();
            pk_stage_rows(cs, codes, i0, (int)min((int64_t)PK_THREADS, n - i0), F1);
            __syncthreads();
        }
        if (i >= n) continue;
        const int32_t *cr = staged ? cs + threadIdx.x * rs : codes + i * F1;
        const uint32_t *mr = mh ? mh + i * F2 : nullptr;
        for (int l = 0; l < L; l++) {
            uint64_t hi = 0, lo = 0;
            for (int k = 0; k < K1; k++) {
                const int f = l * K1 + k;
                const uint32_t v = (uint32_t)((int64_t)cr[f] - (int64_t)fm[f]);
                shl_or(hi, lo, bt[f], v);
            }
            for (int k = 0; k < K2; k++) shl_or(hi, lo, 32, mr[l * K2 + k]);
            klo[(int64_t)l * n + i] = lo;
            if (khi) khi[(int64_t)l * n + i] = hi;
        }
    }
}

// Batched form over the concatenated rows of `count` instances: table l's
// key of global row r (instance i) is i in the bits above `B` followed by
// the instance's own packed K-tuple, so that one sort per table groups every
// instance separately and keeps each instance's lexicographic order.
// (code rows staged through shared memory as in k_pack_keys)
__global__ void __launch_bounds__(PK_THREADS) k_pack_keys_batch(int64_t N, int L, const int32_t *__restrict__ codes,
                                                                int F1, int K1, const int64_t *__restrict__ row_off,
                                                                int count, const int *__restrict__ fmin,
                                                                const int *__restrict__ bits, int B,
                                                                uint64_t *__restrict__ klo,
                                                                uint64_t *__restrict__ khi) {
    extern __shared__ int32_t cs[];
    const bool staged = F1 <= PK_STAGE_MAX;
    const int rs = F1 | 1;
    for (int64_t r0 = (int64_t)blockIdx.x * PK_THREADS; r0 < N; r0 += (int64_t)gridDim.x * PK_THREADS) {
        const int64_t r = r0 + threadIdx.x;
        if (staged) {
            __syncthreads();
            pk_stage_rows(cs, codes, r0, (int)min((int64_t)PK_THREADS, N - r0), F1);
            __syncthreads();
        }
        if (r >= N) continue;
        const int i = find_inst(row_off, count, r);
        const int32_t *cr = staged ? cs + threadIdx.x * rs : codes + r * F1;
        const int *fm = fmin + (int64_t)i * F1;
        const int *bt = bits + (int64_t)i * F1;
        for (int l = 0; l < L; l++) {
            uint64_t hi = 0, lo = 0;
            for (int k = 0; k < K1; k++) {
                const int f = l * K1 + k;
                shl_or(hi, lo, bt[f], (uint32_t)((int64_t)cr[f] - (int64_t)fm[f]));
            }
            const uint64_t iv = (uint64_t)i;
            if (B >= 64) {
                hi |= iv << (B - 64);
            } else if (B > 0) {
                lo |= iv << B;
                hi |= iv >> (64 - B);
            } else {
                lo = iv;
            }
            klo[(int64_t)l * N + r] = lo;
            if (khi) khi[(int64_t)l * N + r] = hi;
        }
    }
}

// E2LSH / SRP row norms of every instance's projections: thread per
// (instance, function)
__global__ void k_row_norms_batch(const ProjArgs *__restrict__ P, int count, int F, float *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)count * F) return;
    const ProjArgs &A = P[e / F];
    const int f = (int)(e % F);
    float s = 0.f;
    for (int j = 0; j < A.d; j++) s = fmaf(A.a[(int64_t)f * A.d + j], A.a[(int64_t)f * A.d + j], s);
    out[e] = sqrtf(s) * 1.0001f;
}

__global__ void k_fill_i32(int *p, int n, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

int grid_for(int64_t work, int threads, int num_sms) {
    int64_t g = ceil_div(work, threads);
    int64_t cap = (int64_t)num_sms * 32;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Thread layout of the projection kernel for F functions.
static void proj_layout(ProjArgs &A, int F) {
    A.F = F;
    A.FPAD = (int)ceil_div(F, PJ_FPT) * PJ_FPT;
    A.FG = A.FPAD / PJ_FPT;
    A.RG = std::max(1, std::min(64, PJ_MAXT / A.FG));  // at most 512 rows per block
}
static int proj_rows(const ProjArgs &A) { return A.RG * PJ_RPT; }
static int proj_threads(const ProjArgs &A) { return (int)ceil_div(A.FG * A.RG, 32) * 32; }  // whole warps
static size_t proj_smem(const ProjArgs &A) { return 2 * (size_t)PJ_KC * (proj_rows(A) + A.FPAD) * sizeof(float); }

geek_status project_dense(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n,
                          int d, const float *a, const float *b, int F, double w, int srp,
                          int32_t *codes, int *fmin, int *fmax, int64_t *n_flagged,
                          int64_t *n_flagged_fp64, cudaStream_t st, int precision) {
    *n_flagged_fp64 = 0;
    if (F > 512) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 512 projections");
    if (d > 100000) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "d > 100000");
    float *anorm;
    GK_TRY(scr.alloc(&anorm, F));
    GK_COUNT();
    k_row_norms<<<(F + 127) / 128, 128, 0, st>>>(a, F, d, anorm);
    GK_COUNT();
    k_fill_i32<<<(F + 255) / 256, 256, 0, st>>>(fmin, F, INT32_MAX);
    GK_COUNT();
    k_fill_i32<<<(F + 255) / 256, 256, 0, st>>>(fmax, F, INT32_MIN);
    GK_LAUNCH(ctx);
    if (n == 0) {
        *n_flagged = 0;
        return GEEK_OK;
    }
    ProjArgs A{};
    A.x = x; A.ldx = ldx; A.n = n; A.d = d;
    proj_layout(A, F);
    A.a = a; A.b = b; A.anorm = anorm;
    A.w = (float)w; A.inv_w = (float)(1.0 / w); A.wd = w;
    // 1/w must be exact for the FP32 cell test's error model to hold as
    // written; otherwise widen it by one more rounding.
    A.srp = srp; A.codes = codes;
    A.fmin = fmin; A.fmax = fmax;
    A.row_base = 0;
    const int TR = proj_rows(A);
    const int threads = proj_threads(A);
    const size_t smem = proj_smem(A);
    if (smem > 200 * 1024) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "projection tile too large");
    GK_CUDA(ctx, cudaFuncSetAttribute(k_project_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned long long *cnt;
    GK_TRY(scr.alloc(&cnt, 1));
    int *status;
    GK_TRY(scr.alloc(&status, 2));
    GK_CUDA(ctx, cudaMemsetAsync(status, 0, 2 * sizeof(int), st));
    int *tc_err = status + 1;  // bounded waits of the tensor-core kernel
    bool use_tc = precision == GEEK_PREC_BF16X3 && proj_tc_eligible(x, ldx, d, F);
    int64_t *row_off;
    ProjArgs *P;
    GK_TRY(scr.alloc(&row_off, 2));
    GK_TRY(scr.alloc(&P, 1));
    const int64_t h_off[2] = {0, n};
    GK_CUDA(ctx, cudaMemcpyAsync(row_off, h_off, sizeof h_off, cudaMemcpyHostToDevice, st));
    int64_t cap = std::max<int64_t>(1 << 20, n * F / 16);
    for (int attempt = 0; attempt < 2; attempt++) {
        uint64_t *flags;
        GK_TRY(scr.alloc(&flags, cap));
        GK_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
        A.flags = flags; A.n_flags = cnt; A.flag_cap = cap;
        GK_CUDA(ctx, cudaMemcpyAsync(P, &A, sizeof A, cudaMemcpyHostToDevice, st));
        const int64_t blocks = ceil_div(n, TR);
        if (use_tc) {
            EvTimer tk(ctx, "kernel.project_tc", st);
            tk.work = (double)n * (4.0 * d + 4.0 * F);  // algorithmic bytes: x read, codes written
            const geek_status ts = proj_tc_launch(ctx, scr, A, tc_err, st);
            if (ts == GEEK_ERR_UNSUPPORTED) use_tc = false;  // no tensor map for this layout
            else GK_TRY(ts);
        }
        if (!use_tc) {
            EvTimer tk(ctx, "kernel.project_fp32", st);
            tk.work = 2.0 * (double)n * (double)F * (double)d;
            GK_COUNT();
            k_project_fp32<false><<<(unsigned)blocks, threads, smem, st>>>(A, nullptr, nullptr, 1);
            GK_LAUNCH(ctx);
        }
        unsigned long long h_cnt = 0;
        GK_CUDA(ctx, cudaMemcpyAsync(&h_cnt, cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        if (use_tc) {
            int h_err = 0;
            GK_CUDA(ctx, cudaMemcpyAsync(&h_err, tc_err, sizeof h_err, cudaMemcpyDeviceToHost, st));
            GK_CUDA(ctx, cudaStreamSynchronize(st));
            if (h_err) return set_error(ctx, (geek_status)h_err, "tensor-core projection: a bounded wait expired");
        }
        if ((int64_t)h_cnt > cap) {  // list overflowed: rerun with the exact size
            cap = (int64_t)h_cnt;
            continue;
        }
        *n_flagged = (int64_t)h_cnt;
        if (h_cnt) {
            uint64_t *flags2;
            unsigned long long *cnt2;
            GK_TRY(scr.alloc(&flags2, (size_t)h_cnt));
            GK_TRY(scr.alloc(&cnt2, 1));
            GK_CUDA(ctx, cudaMemsetAsync(cnt2, 0, sizeof(unsigned long long), st));
            {
                EvTimer tk(ctx, "kernel.recheck_dot2", st);
                GK_COUNT();
                k_recheck_dot2<<<grid_for((int64_t)h_cnt, 256, ctx->num_sms), 256, 0, st>>>(
                    P, row_off, 1, srp, F, flags, cnt, cap, flags2, cnt2);
                GK_LAUNCH(ctx);
            }
            EvTimer tk(ctx, "kernel.recheck_fp64", st);
            GK_COUNT();
            k_recheck_fp64<<<grid_for((int64_t)h_cnt, 128, ctx->num_sms), 128, 0, st>>>(
                P, row_off, 1, srp, F, flags2, cnt2, (int64_t)h_cnt, status);
            GK_LAUNCH(ctx);
            unsigned long long h2 = 0;
            GK_CUDA(ctx, cudaMemcpyAsync(&h2, cnt2, sizeof h2, cudaMemcpyDeviceToHost, st));
            GK_CUDA(ctx, cudaStreamSynchronize(st));
            tk.work = 2.0 * (double)h2 * (double)d;
            *n_flagged_fp64 = (int64_t)h2;
        }
        int h_status[2] = {0, 0};
        GK_CUDA(ctx, cudaMemcpyAsync(h_status, status, sizeof h_status, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        if (h_status[1]) return set_error(ctx, (geek_status)h_status[1], "tensor-core projection: a bounded wait expired");
        if (h_status[0]) return set_error(ctx, (geek_status)h_status[0], "E2LSH code outside int32");
        return GEEK_OK;
    }
    return set_error(ctx, GEEK_ERR_CUDA, "projection flag list did not converge");
}

geek_status proj_batch_setup(geek_ctx *ctx, std::vector<ProjArgs> &P, const std::vector<DenseInst> &inst, int F,
                             int srp, int32_t *codes, const int64_t *row_off_host, ProjBatchBufs &B) {
    if (F > 512) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 512 projections");
    const int count = (int)inst.size();
    P.assign(count, ProjArgs{});
    std::vector<int64_t> toff(count + 1, 0);
    for (int i = 0; i < count; i++) {
        ProjArgs &A = P[i];
        const DenseInst &I = inst[i];
        A.x = I.x; A.ldx = I.ldx; A.n = I.n; A.d = I.d;
        proj_layout(A, F);
        A.a = I.a; A.b = I.b; A.anorm = B.anorm + (int64_t)i * F;
        A.w = (float)I.w; A.inv_w = (float)(1.0 / I.w); A.wd = I.w;
        A.srp = srp;
        A.codes = codes + row_off_host[i] * F;
        A.fmin = B.fmin + (int64_t)i * F;
        A.fmax = B.fmax + (int64_t)i * F;
        A.flags = B.flags; A.n_flags = B.cnt; A.flag_cap = B.cap;
        A.row_base = row_off_host[i];
        toff[i + 1] = toff[i] + ceil_div(I.n, proj_rows(A));
    }
    B.total_tiles = toff[count];
    if (B.total_tiles > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "batch too large for one launch");
    const size_t smem = proj_smem(P[0]);
    if (smem > 200 * 1024) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "projection tile too large");
    GK_CUDA(ctx, cudaFuncSetAttribute(k_project_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GK_CUDA(ctx, cudaMemcpy(B.P, P.data(), sizeof(ProjArgs) * count, cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(B.tile_off, toff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice));
    return GEEK_OK;
}

geek_status proj_batch_enqueue(geek_ctx *ctx, const ProjArgs &P0, int count, int F, int L, int K, int srp,
                               const ProjBatchBufs &B, cudaStream_t st) {
    GK_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(unsigned long long), st));
    GK_CUDA(ctx, cudaMemsetAsync(B.cnt2, 0, sizeof(unsigned long long), st));
    GK_CUDA(ctx, cudaMemsetAsync(B.status, 0, sizeof(int), st));
    const int CF = count * F;
    GK_COUNT();
    k_fill_i32<<<(CF + 255) / 256, 256, 0, st>>>(B.fmin, CF, INT32_MAX);
    GK_COUNT();
    k_fill_i32<<<(CF + 255) / 256, 256, 0, st>>>(B.fmax, CF, INT32_MIN);
    GK_COUNT();
    k_row_norms_batch<<<(CF + 127) / 128, 128, 0, st>>>(B.P, count, F, B.anorm);
    GK_LAUNCH(ctx);
    if (B.total_tiles > 0) {
        GK_COUNT();
        k_project_fp32<true><<<(unsigned)B.total_tiles, proj_threads(P0), proj_smem(P0), st>>>(P0, B.P, B.tile_off,
                                                                                              count);
        GK_COUNT();
        k_recheck_dot2<<<ctx->num_sms * 8, 256, 0, st>>>(B.P, B.row_off, count, srp, F, B.flags, B.cnt, B.cap,
                                                        B.flags2, B.cnt2);
        GK_COUNT();
        k_recheck_fp64<<<ctx->num_sms * 4, 128, 0, st>>>(B.P, B.row_off, count, srp, F, B.flags2, B.cnt2, B.cap,
                                                        B.status);
        GK_LAUNCH(ctx);
    }
    GK_COUNT();
    k_key_layout<<<count, 256, 0, st>>>(B.fmin, B.fmax, L, K, 0, B.bits, B.tbits, B.status);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status pack_keys_batch(geek_ctx *ctx, int64_t N, int L, const int32_t *codes, int K, const int64_t *row_off,
                            int count, const int *fmin, const int *bits, int B, uint64_t *klo, uint64_t *khi,
                            cudaStream_t st) {
    if (N == 0) return GEEK_OK;
    GK_COUNT();
    const int F1 = K * L;
    const size_t smem = F1 <= PK_STAGE_MAX ? (size_t)PK_THREADS * (F1 | 1) * sizeof(int32_t) : 0;
    GK_CUDA(ctx, cudaFuncSetAttribute(k_pack_keys_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(PK_THREADS * (PK_STAGE_MAX | 1) * sizeof(int32_t))));
    k_pack_keys_batch<<<grid_for(N, PK_THREADS, ctx->num_sms), PK_THREADS, smem, st>>>(N, L, codes, F1, K, row_off,
                                                                                       count, fmin, bits, B, klo, khi);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status minhash_rows(geek_ctx *ctx, int64_t n, const int64_t *off, int row_len,
                         const uint32_t *items, int F, const uint64_t *A, const uint64_t *B,
                         uint32_t *out, cudaStream_t st) {
    if (n == 0) return GEEK_OK;
    if (F > 256) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 256 MinHash functions");
    const int threads = 256;
    const int blocks = grid_for(n * 32, threads, ctx->num_sms);
    const bool fixed = off == nullptr;
#define MH_LAUNCH(FPL)                                                                             \
    do {                                                                                          \
        GK_COUNT();                                                                               \
        if (fixed)                                                                                \
            k_minhash<FPL, true><<<blocks, threads, 0, st>>>(n, off, row_len, items, F, A, B, out, F); \
        else                                                                                      \
            k_minhash<FPL, false><<<blocks, threads, 0, st>>>(n, off, row_len, items, F, A, B, out, F); \
    } while (0)
    if (F <= 32) MH_LAUNCH(1);
    else if (F <= 64) MH_LAUNCH(2);
    else if (F <= 128) MH_LAUNCH(4);
    else MH_LAUNCH(8);
#undef MH_LAUNCH
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status minhash_rows64(geek_ctx *ctx, int64_t n, int row_len, const uint64_t *tokens, int F, const uint64_t *A,
                           const uint64_t *B, uint32_t *out, cudaStream_t st) {
    if (n == 0) return GEEK_OK;
    if (F > 256) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 256 MinHash functions");
    const int blocks = grid_for(n * 32, 256, ctx->num_sms);
#define MH_LAUNCH(FPL)                                                                                             \
    do {                                                                                                          \
        GK_COUNT();                                                                                               \
        k_minhash<FPL, true, uint64_t><<<blocks, 256, 0, st>>>(n, nullptr, row_len, tokens, F, A, B, out, F);    \
    } while (0)
    if (F <= 32) MH_LAUNCH(1);
    else if (F <= 64) MH_LAUNCH(2);
    else if (F <= 128) MH_LAUNCH(4);
    else MH_LAUNCH(8);
#undef MH_LAUNCH
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status key_layout(geek_ctx *ctx, Scratch &scr, const int *fmin, const int *fmax, int L, int K1,
                       int K2, int *bits_dev, std::vector<int> &tbits, cudaStream_t st) {
    int *tb, *status;
    GK_TRY(scr.alloc(&tb, L));
    GK_TRY(scr.alloc(&status, 1));
    GK_CUDA(ctx, cudaMemsetAsync(status, 0, sizeof(int), st));
    GK_COUNT();
    k_key_layout<<<1, 256, 0, st>>>(fmin, fmax, L, K1, K2, bits_dev, tb, status);
    GK_LAUNCH(ctx);
    tbits.assign(L, 0);
    int h_status = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(tbits.data(), tb, sizeof(int) * L, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_status) return set_error(ctx, GEEK_ERR_OVERFLOW, "a table key needs more than 128 bits");
    return GEEK_OK;
}

geek_status pack_keys(geek_ctx *ctx, int64_t n, int L, const int32_t *codes, int F1, int K1,
                      const int *fmin, const int *bits, const uint32_t *mh, int F2, int K2,
                      uint64_t *klo, uint64_t *khi, cudaStream_t st) {
    if (n == 0) return GEEK_OK;
    GK_COUNT();
    const size_t smem = (F1 > 0 && F1 <= PK_STAGE_MAX) ? (size_t)PK_THREADS * (F1 | 1) * sizeof(int32_t) : 0;
    GK_CUDA(ctx, cudaFuncSetAttribute(k_pack_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(PK_THREADS * (PK_STAGE_MAX | 1) * sizeof(int32_t))));
    k_pack_keys<<<grid_for(n, PK_THREADS, ctx->num_sms), PK_THREADS, smem, st>>>(n, L, codes, F1, K1, fmin, bits, mh,
                                                                                 F2, K2, klo, khi);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}

geek_status group_tables(geek_ctx *ctx, Scratch &scr, int64_t n, int L, uint64_t *klo,
                         uint64_t *khi, int nbits, uint32_t *ids, int32_t *obj_bucket,
                         int64_t **boff_out, std::vector<int64_t> &nb, int64_t *NB_out,
                         cudaStream_t st) {
    launch_iota_u32(ids, n * L, n, st);
    GK_LAUNCH(ctx);
    {
        EvTimer tk(ctx, "hash.sort", st);
        GK_TRY(radix_sort_segments(ctx, scr, L, n, &klo, khi ? &khi : nullptr, &ids, nbits, st));
    }
    return segment_buckets(ctx, scr, L, n, klo, nbits > 64 ? khi : nullptr, ids, obj_bucket, boff_out, nb, NB_out,
                           st);
}
