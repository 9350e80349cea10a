// Allocation-free variant of the dense FP32 assignment (geek_assign_centers
// with GEEK_PREC_FP32) for callers that must not allocate device memory.
//
// Its scratch (the FP32 copy of the centres, their squared norms and the
// bound on their norms) lives in one file-scope device array of fixed size
// that every GPU loading this library holds until the process exits.  Rows
// whose argmin is uncertain are marked in the caller's label array itself
// (value -2) and decided in FP64 by a second kernel, so no per-row scratch is
// needed.  The results equal geek_assign_centers'.
#include <cfloat>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t NA_SCRATCH_BYTES = (size_t)GEEK_NOALLOC_MAX_KD * 4 + (size_t)GEEK_NOALLOC_MAX_K * 4 + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_TR = 128, NA_TC = 64, NA_KC = 32, NA_RPT = 8, NA_CPT = 4;
constexpr int32_t NA_UNDECIDED = -2;

struct NaLayout {
    float *c32;         // k x d
    float *cn;          // k
    unsigned *cmax;     // 1 (bits of a non-negative float)
};

__host__ __device__ inline NaLayout na_layout(unsigned char *base) {
    NaLayout L;
    L.c32 = (float *)base;
    L.cn = (float *)(base + (size_t)GEEK_NOALLOC_MAX_KD * 4);
    L.cmax = (unsigned *)(base + (size_t)GEEK_NOALLOC_MAX_KD * 4 + (size_t)GEEK_NOALLOC_MAX_K * 4);
    return L;
}

__global__ void k_na_clear(unsigned *cmax) { *cmax = 0u; }

__global__ void k_na_prep(const double *__restrict__ c64, int64_t k, int d, NaLayout S) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < d; t++) {
            const double v = c64[j * d + t];
            S.c32[j * d + t] = (float)v;
            s += v * v;
        }
        S.cn[j] = (float)s;
        atomicMax(S.cmax, __float_as_uint((float)sqrt(s) * (1.f + 1e-6f)));
    }
}

struct NaBest {
    float b1, b2;
    int i1;
};

__device__ __forceinline__ void na_push(NaBest &B, float v, int j) {
    if (v < B.b1) {
        B.b2 = B.b1;
        B.b1 = v;
        B.i1 = j;
    } else {
        B.b2 = fminf(B.b2, v);
    }
}

__device__ __forceinline__ NaBest na_merge(NaBest a, NaBest b) {
    NaBest r;
    const bool tb = b.b1 < a.b1 || (b.b1 == a.b1 && b.i1 < a.i1);
    r.b1 = tb ? b.b1 : a.b1;
    r.i1 = tb ? b.i1 : a.i1;
    r.b2 = fminf(fminf(a.b2, b.b2), tb ? a.b1 : b.b1);
    return r;
}

// FP32 SIMT pass: certain rows get their label, the others NA_UNDECIDED
__global__ void __launch_bounds__(256) k_na_assign(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                                   int64_t k, NaLayout S, int32_t *__restrict__ labels) {
    extern __shared__ float sm[];
    float *xs = sm;                      // [d][NA_TR]
    float *cs = sm + (size_t)d * NA_TR;  // [NA_KC][NA_TC]
    __shared__ float cns[NA_TC];
    const float cmax = __uint_as_float(*S.cmax);
    const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * NA_TR;
    for (int e = t; e < NA_TR * d; e += 256) {
        const int r = e / d, kk = e % d;
        const int64_t row = row0 + r;
        xs[kk * NA_TR + r] = row < n ? x[row * ldx + kk] : 0.f;
    }
    NaBest B[NA_RPT];
#pragma unroll
    for (int r = 0; r < NA_RPT; r++) B[r] = NaBest{FLT_MAX, FLT_MAX, 0x7FFFFFFF};
    for (int64_t j0 = 0; j0 < k; j0 += NA_TC) {
        float acc[NA_RPT][NA_CPT];
#pragma unroll
        for (int r = 0; r < NA_RPT; r++)
#pragma unroll
            for (int c = 0; c < NA_CPT; c++) acc[r][c] = 0.f;
        for (int k0 = 0; k0 < d; k0 += NA_KC) {
            __syncthreads();
            for (int e = t; e < NA_TC * NA_KC; e += 256) {
                const int c = e / NA_KC, kk = e % NA_KC;
                const int64_t j = j0 + c;
                cs[kk * NA_TC + c] = (j < k && k0 + kk < d) ? S.c32[j * d + k0 + kk] : 0.f;
            }
            if (k0 == 0 && t < NA_TC) cns[t] = j0 + t < k ? S.cn[j0 + t] : FLT_MAX;
            __syncthreads();
            const int kmax = min(NA_KC, d - k0);
            for (int kk = 0; kk < kmax; kk++) {
                const float4 x0 = *reinterpret_cast<const float4 *>(&xs[(k0 + kk) * NA_TR + rg * NA_RPT]);
                const float4 x1 = *reinterpret_cast<const float4 *>(&xs[(k0 + kk) * NA_TR + rg * NA_RPT + 4]);
                const float4 cv = *reinterpret_cast<const float4 *>(&cs[kk * NA_TC + cg * NA_CPT]);
                const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                for (int r = 0; r < NA_RPT; r++)
#pragma unroll
                    for (int c = 0; c < NA_CPT; c++) acc[r][c] = fmaf(xv[r], cc[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int c = 0; c < NA_CPT; c++) {
            const int64_t j = j0 + cg * NA_CPT + c;
            if (j >= k) continue;
            const float cnj = cns[cg * NA_CPT + c];
#pragma unroll
            for (int r = 0; r < NA_RPT; r++) na_push(B[r], fmaf(-2.f, acc[r][c], cnj), (int)j);
        }
    }
#pragma unroll
    for (int r = 0; r < NA_RPT; r++) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            NaBest q;
            q.b1 = __shfl_xor_sync(0xffffffffu, B[r].b1, o);
            q.b2 = __shfl_xor_sync(0xffffffffu, B[r].b2, o);
            q.i1 = __shfl_xor_sync(0xffffffffu, B[r].i1, o);
            B[r] = na_merge(B[r], q);
        }
    }
    if (cg == 0) {
#pragma unroll
        for (int r = 0; r < NA_RPT; r++) {
            const int64_t row = row0 + rg * NA_RPT + r;
            if (row >= n) continue;
            float xs2 = 0.f;
            for (int kk = 0; kk < d; kk++) {
                const float v = xs[kk * NA_TR + rg * NA_RPT + r];
                xs2 = fmaf(v, v, xs2);
            }
            const float W = 2.f * window_fp32(sqrtf(xs2) * (1.f + 1.0e-3f), cmax, d);
            const bool valid = B[r].i1 != 0x7FFFFFFF;
            const bool sure = valid && (k == 1 || (B[r].b2 - B[r].b1 > W * (1.f + 1e-6f)));
            labels[row] = sure ? B[r].i1 : NA_UNDECIDED;
        }
    }
}

// FP64 decision of every row marked NA_UNDECIDED (block per row, grid-stride)
__global__ void __launch_bounds__(256) k_na_decide(const float *__restrict__ x, int64_t ldx, int64_t n, int d,
                                                   const double *__restrict__ c64, int64_t k, NaLayout S,
                                                   int32_t *__restrict__ labels) {
    extern __shared__ float xr[];
    __shared__ float red_f[256];
    __shared__ double red_d[256];
    __shared__ int red_i[256];
    const int t = threadIdx.x;
    const float cmax = __uint_as_float(*S.cmax);
    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        if (labels[row] != NA_UNDECIDED) continue;  // uniform across the block
        __syncthreads();
        for (int kk = t; kk < d; kk += 256) xr[kk] = x[row * ldx + kk];
        __syncthreads();
        float xs2 = 0.f;
        for (int kk = 0; kk < d; kk++) xs2 = fmaf(xr[kk], xr[kk], xs2);
        const float xn = sqrtf(xs2) * (1.f + 1.0e-3f);
        float m = FLT_MAX;
        for (int64_t j = t; j < k; j += 256) {
            float dot = 0.f;
            for (int kk = 0; kk < d; kk++) dot = fmaf(xr[kk], S.c32[j * d + kk], dot);
            m = fminf(m, fmaf(-2.f, dot, S.cn[j]));
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
            for (int kk = 0; kk < d; kk++) dot = fmaf(xr[kk], S.c32[j * d + kk], dot);
            if (fmaf(-2.f, dot, S.cn[j]) <= lim) {
                const double D = ref_dist(xr, c64 + j * d, d);
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
        if (t == 0) labels[row] = red_i[0] == 0x7FFFFFFF ? -1 : red_i[0];
        __syncthreads();
    }
}

// per-device set-up: device address of the scratch array and the kernels'
// shared-memory limit (done once, with that device current)
struct NaDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;
    int num_sms = 0;
};
std::mutex g_na_mutex;
NaDevice g_na_dev[64];

geek_status na_setup(int dev, NaDevice **out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (dev < 0 || dev >= 64) return GEEK_ERR_UNSUPPORTED;
    NaDevice &D = g_na_dev[dev];
    if (!D.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GEEK_ERR_CUDA;
        }
        const int smem_max = 256 * NA_TR * (int)sizeof(float) + NA_KC * NA_TC * (int)sizeof(float);
        if (cudaFuncSetAttribute(k_na_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
            cudaDeviceGetAttribute(&D.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return GEEK_ERR_CUDA;
        }
        D.scratch = (unsigned char *)p;
        D.ready = true;
    }
    *out = &D;
    return GEEK_OK;
}

}  // namespace

extern "C" geek_status geek_assign_centers_noalloc(const float *x, int64_t n, int32_t d, int64_t ldx,
                                                   const double *centers, int64_t k, int32_t *labels,
                                                   geek_stream stream) {
    if (n < 0 || d < 1 || ldx < d || k < 1 || (n > 0 && (!x || !labels)) || !centers) return GEEK_ERR_INVALID;
    if (d > 256 || k > GEEK_NOALLOC_MAX_K || k * (int64_t)d > GEEK_NOALLOC_MAX_KD || n > 0x7FFFFFFFLL)
        return GEEK_ERR_UNSUPPORTED;
    // an error left by earlier work on this thread belongs to that work:
    // report it without clearing it instead of launching behind it
    if (cudaPeekAtLastError() != cudaSuccess) return GEEK_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GEEK_ERR_CUDA;
    }
    NaDevice *D;
    geek_status s = na_setup(dev, &D);
    if (s != GEEK_OK) return s;
    if (n == 0) return GEEK_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const NaLayout S = na_layout(D->scratch);
    // each launch is checked on its own, so an error this call reports is
    // its own (an error pending from earlier work was refused on entry)
    GK_COUNT();
    k_na_clear<<<1, 1, 0, st>>>(S.cmax);
    if (cudaGetLastError() != cudaSuccess) return GEEK_ERR_CUDA;
    GK_COUNT();
    k_na_prep<<<(int)std::min<int64_t>(ceil_div(k, 128), (int64_t)D->num_sms * 8), 128, 0, st>>>(centers, k, d, S);
    if (cudaGetLastError() != cudaSuccess) return GEEK_ERR_CUDA;
    const size_t smem = (size_t)d * NA_TR * sizeof(float) + (size_t)NA_KC * NA_TC * sizeof(float);
    GK_COUNT();
    k_na_assign<<<(unsigned)ceil_div(n, NA_TR), 256, smem, st>>>(x, ldx, n, d, k, S, labels);
    if (cudaGetLastError() != cudaSuccess) return GEEK_ERR_CUDA;
    GK_COUNT();
    k_na_decide<<<(int)std::min<int64_t>(n, (int64_t)D->num_sms * 8), 256, d * sizeof(float), st>>>(x, ldx, n, d,
                                                                                                   centers, k, S, labels);
    if (cudaGetLastError() != cudaSuccess) return GEEK_ERR_CUDA;
    return GEEK_OK;
}
