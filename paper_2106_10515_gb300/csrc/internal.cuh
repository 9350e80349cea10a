// Host-side entry points shared between translation units.
#pragma once
#include <vector>

#include "common.cuh"


// ---- dense assignment arithmetic (assign.cu, noalloc.cu) -----------------
// Both assignment entry points promise the same labels, so the reference
// distance and the FP32 window they decide with are defined once, here.

// FP64 reference distance of the pinned definition.
static __device__ __forceinline__ double ref_dist(const float *__restrict__ x, const double *__restrict__ c, int d) {
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
static __device__ __forceinline__ float window_fp32(float xn, float cmax, int d) {
    const float u = 5.9604645e-8f;
    const float gam = (float)d * u / (1.f - (float)d * u);
    const float e32 = (2.f * gam + 4.f * u) * xn * cmax + 2.f * u * cmax * cmax;
    const float s = xn + cmax;
    const float e64 = (float)(d + 3) * 1.1102230e-16f * s * s;
    return 1.01f * (e32 + e64) + 1e-30f;
}


// ---- dense projection (hash.cu) -------------------------------------------
// Per-instance arguments of the FP32 projection kernel and its recheck
// stages (device copies are read by the batched kernels).
struct ProjArgs {
    const float *x;
    int64_t ldx;
    int64_t n;
    int d;
    int F, FPAD, FG, RG;  // functions, padded to 8, function groups, row groups
    const float *a;       // F x d
    const float *b;       // F
    const float *anorm;   // F
    float w, inv_w;
    int srp;
    int32_t *codes;       // n x F
    uint64_t *flags;      // (row << 16 | f)
    unsigned long long *n_flags;
    int64_t flag_cap;
    int *fmin, *fmax;     // F
    double wd;            // w as given (the reference divides by it in FP64)
    int64_t row_base;     // global row of local row 0 (flag list entries)
};

// One dense instance of a batch (device pointers).
struct DenseInst {
    const float *x;
    int64_t ldx, n;
    int d;
    const float *a, *b;
    double w;
};

// Device buffers of the batched hash phase (owned by the batch plan).
struct ProjBatchBufs {
    ProjArgs *P = nullptr;         // count
    int64_t *tile_off = nullptr;   // count + 1: projection blocks per instance
    int64_t *row_off = nullptr;    // count + 1: global rows per instance
    float *anorm = nullptr;        // count * F
    int *fmin = nullptr, *fmax = nullptr, *bits = nullptr;  // count * F
    int *tbits = nullptr;          // count * L
    uint64_t *flags = nullptr, *flags2 = nullptr;           // cap
    unsigned long long *cnt = nullptr, *cnt2 = nullptr;
    int *status = nullptr;
    int64_t cap = 0;
    int64_t total_tiles = 0;
};

geek_status proj_batch_setup(geek_ctx *ctx, std::vector<ProjArgs> &P, const std::vector<DenseInst> &inst, int F,
                             int srp, int32_t *codes, const int64_t *row_off_host, ProjBatchBufs &B);
// Enqueues the whole batched hash phase up to the key layouts; no host
// synchronisation and no allocation, so it can be captured in a CUDA graph.
geek_status proj_batch_enqueue(geek_ctx *ctx, const ProjArgs &P0, int count, int F, int L, int K, int srp,
                               const ProjBatchBufs &B, cudaStream_t st);
geek_status pack_keys_batch(geek_ctx *ctx, int64_t N, int L, const int32_t *codes, int K, const int64_t *row_off,
                            int count, const int *fmin, const int *bits, int B, uint64_t *klo, uint64_t *khi,
                            cudaStream_t st);

// hash.cu
// precision GEEK_PREC_FP32: FP32 SIMT projection; GEEK_PREC_BF16X3: the
// three-term split BF16 tcgen05 projection (proj_tc.cu) where eligible.
geek_status project_dense(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n,
                          int d, const float *a, const float *b, int F, double w, int srp,
                          int32_t *codes, int *fmin, int *fmax, int64_t *n_flagged,
                          int64_t *n_flagged_fp64, cudaStream_t st, int precision = GEEK_PREC_FP32);
// proj_tc.cu: shapes the tensor-core projection takes (d <= 128, F <= 128,
// 16-byte aligned rows), and one launch of it with the arguments of the
// FP32 kernel (codes, min / max, flag list); err: device word for timeouts.
bool proj_tc_eligible(const float *x, int64_t ldx, int d, int F);
geek_status proj_tc_launch(geek_ctx *ctx, Scratch &scr, const ProjArgs &P, int *err, cudaStream_t st);
// MinHash of fixed rows of 64-bit tokens (a DOPH reduction): out n x F.
geek_status minhash_rows64(geek_ctx *ctx, int64_t n, int row_len, const uint64_t *tokens, int F, const uint64_t *A,
                           const uint64_t *B, uint32_t *out, cudaStream_t st);
// DOPH reduction of CSR sets (doph.cu): tokens n x Dp, 1 <= Dp <= 1024.
geek_status doph_reduce(geek_ctx *ctx, int64_t n, const int64_t *off, const uint32_t *items, int Dp, uint64_t Ap,
                        uint64_t Bp, uint64_t *tokens, cudaStream_t st);
geek_status minhash_rows(geek_ctx *ctx, int64_t n, const int64_t *off, int row_len,
                         const uint32_t *items, int F, const uint64_t *A, const uint64_t *B,
                         uint32_t *out, cudaStream_t st);
geek_status key_layout(geek_ctx *ctx, Scratch &scr, const int *fmin, const int *fmax, int L, int K1,
                       int K2, int *bits_dev, std::vector<int> &tbits, cudaStream_t st);
geek_status pack_keys(geek_ctx *ctx, int64_t n, int L, const int32_t *codes, int F1, int K1,
                      const int *fmin, const int *bits, const uint32_t *mh, int F2, int K2,
                      uint64_t *klo, uint64_t *khi, cudaStream_t st);
// Alg. 1 (qalsh.cu): m tables of t buckets from the m QALSH projections.
geek_status hash_qalsh(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d, const float *a,
                       int m, int t, geek_buckets *b, cudaStream_t st);
geek_status group_tables(geek_ctx *ctx, Scratch &scr, int64_t n, int L, uint64_t *klo,
                         uint64_t *khi, int nbits, uint32_t *ids, int32_t *obj_bucket,
                         int64_t **boff_out, std::vector<int64_t> &nb, int64_t *NB_out,
                         cudaStream_t st);
int grid_for(int64_t work, int threads, int num_sms);

// Library-owned result of geek_hash.
struct geek_buckets {
    geek_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;     // stream of creation: allocations and frees are ordered on it
    int kind = 0;
    int64_t n = 0;
    int L = 0, K = 0, Kc = 0, F = 0;
    int key_bits_max = 0;
    int64_t NB = 0;
    int64_t n_flagged = 0;       // elements outside the FP32 certainty window
    int64_t n_flagged_fp64 = 0;  // of those, elements decided by the FP64 reference
    std::vector<int64_t> nb;       // buckets per table
    int32_t *obj_bucket = nullptr; // L x n
    int64_t *boff = nullptr;       // NB + 1
    uint32_t *members = nullptr;   // L x n
    int32_t *codes = nullptr;      // n x F (E2LSH codes, or MinHash values for SETS)
    // HETERO: per table, the packed key of the numeric E2LSH part only (the
    // unified categorical attribute used for assignment), L x n
    uint64_t *num_key = nullptr;
    // SETS hashed through DOPH: the D' tokens of every object, n x D'
    uint64_t *doph_tok = nullptr;
    int doph_bins = 0;
};

struct silk_seeds {
    geek_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;  // stream of creation (allocations and frees)
    int64_t k = 0, n_ids = 0, n_multiset = 0;
    int64_t *off = nullptr;  // k + 1
    int32_t *ids = nullptr;  // n_ids
};

// silk.cu
// Batched instances: object ids are global rows, instance i owning
// [row_off[i], row_off[i + 1]) (device, count + 1).  SILK then runs on every
// instance at once with bins never spanning instances and each instance's
// own coefficients (instance-major: Ls*Ks SILK pairs, Ks dedup pairs each)
// applied to its local ids, which gives each instance's own seeds.
struct SilkBatch {
    const int64_t *row_off = nullptr;
    int count = 1;
    // set inside silk_run: per-instance slot regions of the grouping tables,
    // for all sets and (_m) for the sets of two or more objects
    const int64_t *slot_off = nullptr, *slot_cap = nullptr;
    int64_t slots = 0;
    const int64_t *slot_off_m = nullptr, *slot_cap_m = nullptr;
    int64_t slots_m = 0;
    const uint32_t *set_inst = nullptr;  // instance of every virtual bucket
};
geek_status silk_run(geek_ctx *ctx, const geek_buckets *b, const silk_params *p, silk_seeds *out,
                     cudaStream_t st, const SilkBatch *bt = nullptr);

// tc_assign.cu
// One instance of a (batched) BF16 tcgen05 assignment: rows x (n x d,
// stride ldx) against k FP64 centres, labels written at labels[0..n), flag
// list entries are row_base + local row; N = centre-tile width (64/128/256).
struct TcPlanInst {
    const float *x;
    int64_t ldx, n;
    int d;
    const double *centres;
    int64_t k;
    int32_t *labels;
    int64_t row_base;
    int N;
    int split;  // 1: split-BF16 (three products, narrow window); needs N * Kp <= 8192
};
struct TcInst;
struct TcXPrep;
struct TcCPrep;
// Buffers, descriptors and the unit list (instance, row tile) of one
// persistent tcgen05 launch over a set of instances.
struct TcPlan {
    struct Impl;
    Impl *impl = nullptr;
    std::vector<TcPlanInst> desc;
    int count = 0;
    int64_t N_total = 0, kpad_total = 0, nunits = 0, nunits_x3 = 0;
    bool allow_split = false;    // buffers sized for the split layout of every instance
    int2 *tune_units = nullptr;  // scratch unit list of tc_plan_launch_subset
    int64_t tune_cap = 0;
    TcInst *inst = nullptr;
    TcXPrep *xprep = nullptr;
    TcCPrep *cprep = nullptr;
    int2 *units = nullptr;
    int64_t *row_off = nullptr, *kpad_off_dev = nullptr;
    float *xnorm = nullptr;
    unsigned *cmax_bits = nullptr;
    int *err = nullptr;
    std::vector<void *> owned;
};
// scr == nullptr: buffers are cudaMalloc'd and owned by the plan
geek_status tc_plan_build(geek_ctx *ctx, Scratch *scr, const std::vector<TcPlanInst> &desc, TcPlan *P,
                          cudaStream_t st);
// conversions of X and the centres (BF16, norms, max |c|^2)
geek_status tc_plan_convert(geek_ctx *ctx, const TcPlan &P, cudaStream_t st);
// the persistent tcgen05 pass (after tc_plan_convert); n_flag zeroed by the caller
geek_status tc_plan_launch(geek_ctx *ctx, const TcPlan &P, int32_t *flag_rows, unsigned long long *n_flag,
                           cudaStream_t st);
geek_status tc_plan_enqueue(geek_ctx *ctx, const TcPlan &P, int32_t *flag_rows, unsigned long long *n_flag,
                            cudaStream_t st);
geek_status tc_plan_upload(geek_ctx *ctx, TcPlan *P, cudaStream_t st);
geek_status tc_plan_set_modes(geek_ctx *ctx, TcPlan *P, const std::vector<int> &N, const std::vector<int> &split,
                              cudaStream_t st);
geek_status tc_plan_launch_subset(geek_ctx *ctx, TcPlan *P, const std::vector<int> &which, int32_t *flag_rows,
                                  unsigned long long *n_flag, cudaStream_t st);
geek_status tc_plan_check(geek_ctx *ctx, const TcPlan &P, cudaStream_t st);
void tc_plan_free(TcPlan *P);
int tc_tile_candidates(const int **tiles);
geek_status assign_tc_bf16(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                           const double *centres, int64_t k, int split, int32_t *labels, int32_t *flag_rows,
                           unsigned long long *n_flag, cudaStream_t st);

// assign.cu
// Centre preparation of one instance (device copies): FP32 copy and |c|^2
// of centres k_base.. (global index) and the max of |c| (FP32 bits).
struct CInst {
    const double *c64;
    float *c32;
    float *cn;
    unsigned *cmax_bits;
    int d;
    int64_t k_base;
};
// FP64 argmin decision of one instance's flagged rows (device copies).
struct RInst {
    const float *x;
    int64_t ldx;
    int d;
    const float *c32, *cn;
    const double *c64;
    int64_t k;
    const unsigned *cmax_bits;
    int32_t *labels;
    int64_t row_base;
};
// Centroids of one instance's seeds (device copies): seeds seed_base ..
// seed_base + k - 1 of the global seed list, member ids global rows.
struct CenInst {
    const float *x;
    int64_t ldx;
    int d;
    int64_t row_base, seed_base;
    double *c;
};
// SSE / radius of one instance (device copies).
struct SInst {
    const float *x;
    int64_t ldx, n;
    int d;
    const float *chi, *clo;
    int64_t k;
    const int32_t *labels;
};
// Enqueue-only batched steps (no host synchronisation, no allocation).
geek_status centroids_batch(geek_ctx *ctx, const CenInst *C, const int64_t *seed_inst_off, int count, int64_t ktot,
                            int dmax, const int64_t *soff, const int32_t *sids, cudaStream_t st);
geek_status centre_prep_batch(geek_ctx *ctx, const CInst *C, const int64_t *k_off, int count, int64_t ktot,
                              cudaStream_t st);
geek_status centre_split(geek_ctx *ctx, const double *c64, int64_t total, float *chi, float *clo, cudaStream_t st);
geek_status stats_batch(geek_ctx *ctx, const SInst *S, const int2 *units, int64_t nunits, const int64_t *unit_off,
                        int count, double *part_sum, float *part_max, double *sse, double *rmax, cudaStream_t st);
geek_status fill_labels(geek_ctx *ctx, int32_t *labels, int64_t n, int32_t v, cudaStream_t st);
// Buffers of decide_flags (scratch-owned when allocated from a Scratch).
struct DecideBufs {
    int *cnt = nullptr;            // count: flagged rows per instance
    int64_t *cursor = nullptr;     // count
    int *unit_inst = nullptr;      // units of up to 128 flagged rows
    int64_t *unit_start = nullptr;
    int *unit_cnt = nullptr;
    int *n_units = nullptr;
    int32_t *grows = nullptr;      // flagged rows grouped by instance
    int32_t *flags2 = nullptr;     // rows left to the FP64 reference
    float *flags2_m = nullptr;     // their smallest FP32 value (NaN: none)
    float *mrow = nullptr;         // the same value by global row
    unsigned long long *n_flag2 = nullptr;
    std::vector<void *> owned;
};
geek_status decide_bufs_alloc(geek_ctx *ctx, Scratch *scr, int count, int64_t n_total, DecideBufs &B);
void decide_bufs_free(DecideBufs &B);
geek_status decide_flags(geek_ctx *ctx, const RInst *R, const int64_t *row_off, int count, int dmax,
                         const int32_t *flags, const unsigned long long *n_flag, const DecideBufs &B,
                         cudaStream_t st);
geek_status assign_dense_centres(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx,
                                 int64_t n, int d, const double *centres, int64_t k, int precision,
                                 int32_t *labels, geek_assign_stats *stats, cudaStream_t st);
geek_status cluster_radius(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                           const double *centres, int64_t k, const int32_t *labels, double *radius, cudaStream_t st);
// Sect. 5's extra passes: per pass, centre j <- FP64 mean of the objects
// labelled j (unchanged without members), then the exact reassignment.
geek_status refine_dense(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d, double *centres,
                         int64_t k, int passes, int precision, int32_t *labels, geek_assign_stats *stats,
                         cudaStream_t st);
geek_status centroids_from_seeds(geek_ctx *ctx, const float *x, int64_t ldx, int d,
                                 const silk_seeds *s, double *centres, cudaStream_t st);
// Library-owned central vectors of one assignment (geek_assign_ex).
struct geek_centres {
    geek_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;     // stream of creation (allocations and frees)
    int kind = 0;
    int64_t k = 0;
    int d = 0, n_attr = 0;
    int64_t n_items = 0;
    double *centers = nullptr;     // DENSE: k x d
    int64_t *modes = nullptr;      // HETERO: k x n_attr
    int64_t *item_off = nullptr;   // SETS: k + 1
    uint32_t *items = nullptr;     // SETS: n_items
};
// Stream-ordered allocation of a result handle's buffer (NOMEM on failure).
geek_status own_alloc(geek_ctx *ctx, void **p, size_t bytes, cudaStream_t st);
// keep (nullable): receives the central vectors the assignment used.
// Sets reduced by DOPH (b->doph_bins > 0): per-dimension modes, Jaccard of tokens.
geek_status assign_doph(geek_ctx *ctx, Scratch &scr, const geek_buckets *b, const silk_seeds *s, int32_t *labels,
                        geek_assign_stats *stats, geek_centres *keep, cudaStream_t st);
geek_status assign_hetero(geek_ctx *ctx, Scratch &scr, const geek_buckets *b, const uint32_t *tok,
                          int n_cat, const silk_seeds *s, int32_t *labels, geek_assign_stats *stats,
                          geek_centres *keep, cudaStream_t st);
geek_status assign_sets(geek_ctx *ctx, Scratch &scr, const int64_t *off, const uint32_t *items,
                        int64_t n, const silk_seeds *s, int32_t *labels, geek_assign_stats *stats,
                        geek_centres *keep, cudaStream_t st);
