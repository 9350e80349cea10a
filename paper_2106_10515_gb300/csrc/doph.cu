// DOPH reduction, the first step of the sparse transform (Alg. 3): densified
// one permutation hashing with rotation (Shrivastava and Li).  One hash
// pi(v) = h(Ap, Bp, v) stands for the permutation; its 32-bit range is cut
// into Dp equal bins, bin(v) = (pi(v) * Dp) >> 32 and offset(v) =
// (pi(v) * Dp) mod 2^32; a bin keeps the smallest offset of its items; an
// empty bin takes the value of the first non-empty bin to its right
// (circular) at distance t; an empty set gives t = Dp and value 2^32 - 1.
// The reduced object is the set of Dp tokens (b << 48) | (t << 32) | value.
#include "internal.cuh"

namespace {

constexpr int DP_MAX = 1024, DP_WARPS = 8;

// warp per set: bin minima by shared-memory atomics, then lane 0 finds for
// every bin the nearest non-empty bin at or to its right (walking the bins
// twice around from the end), then the lanes write the tokens
__global__ void __launch_bounds__(DP_WARPS * 32) k_doph(int64_t n, const int64_t *__restrict__ off,
                                                     const uint32_t *__restrict__ items, int Dp, uint64_t Ap,
                                                     uint64_t Bp, uint64_t *__restrict__ tokens) {
    extern __shared__ unsigned long long dsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long *m = dsm + (size_t)wib * Dp;
    int *nxt = (int *)(dsm + (size_t)DP_WARPS * Dp) + (size_t)wib * Dp;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nw) {
        for (int b = lane; b < Dp; b += 32) m[b] = ~0ull;
        __syncwarp();
        for (int64_t p = off[i] + lane; p < off[i + 1]; p += 32) {
            const uint64_t sc = (uint64_t)mh_hash32(Ap, Bp, items[p]) * (uint64_t)Dp;
            atomicMin(&m[sc >> 32], (unsigned long long)(sc & 0xFFFFFFFFull));
        }
        __syncwarp();
        if (lane == 0) {
            int last = -1;  // nearest non-empty index (0 .. 2Dp-1) at or right of b
            for (int b = 2 * Dp - 1; b >= 0; b--) {
                if (m[b % Dp] != ~0ull) last = b;
                if (b < Dp) nxt[b] = last;
            }
        }
        __syncwarp();
        for (int b = lane; b < Dp; b += 32) {
            uint64_t t, v;
            if (nxt[b] < 0) {
                t = (uint64_t)Dp;
                v = 0xFFFFFFFFull;
            } else {
                t = (uint64_t)(nxt[b] - b);
                v = m[nxt[b] % Dp];
            }
            tokens[i * Dp + b] = ((uint64_t)b << 48) | (t << 32) | v;
        }
        __syncwarp();  // m and nxt are reused by the next set
    }
}

}  // namespace

geek_status doph_reduce(geek_ctx *ctx, int64_t n, const int64_t *off, const uint32_t *items, int Dp, uint64_t Ap,
                        uint64_t Bp, uint64_t *tokens, cudaStream_t st) {
    if (Dp < 1 || Dp > DP_MAX) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "DOPH: 1 <= bins <= 1024");
    if (n == 0) return GEEK_OK;
    const size_t smem = (size_t)DP_WARPS * Dp * (sizeof(unsigned long long) + sizeof(int));
    GK_CUDA(ctx, cudaFuncSetAttribute(k_doph, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GK_COUNT();
    k_doph<<<(unsigned)std::min<int64_t>(ceil_div(n, DP_WARPS), (int64_t)ctx->num_sms * 8), DP_WARPS * 32, smem, st>>>(
        n, off, items, Dp, Ap, Bp, tokens);
    GK_LAUNCH(ctx);
    return GEEK_OK;
}
