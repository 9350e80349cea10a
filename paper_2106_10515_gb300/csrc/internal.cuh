// Host-side entry points shared between translation units.
#pragma once
#include <vector>

#include "common.cuh"

// hash.cu
geek_status project_dense(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n,
                          int d, const float *a, const float *b, int F, double w, int srp,
                          int32_t *codes, int *fmin, int *fmax, int64_t *n_flagged,
                          int64_t *n_flagged_fp64, cudaStream_t st);
geek_status minhash_rows(geek_ctx *ctx, int64_t n, const int64_t *off, int row_len,
                         const uint32_t *items, int F, const uint64_t *A, const uint64_t *B,
                         uint32_t *out, cudaStream_t st);
geek_status key_layout(geek_ctx *ctx, Scratch &scr, const int *fmin, const int *fmax, int L, int K1,
                       int K2, int *bits_dev, std::vector<int> &tbits, cudaStream_t st);
geek_status pack_keys(geek_ctx *ctx, int64_t n, int L, const int32_t *codes, int F1, int K1,
                      const int *fmin, const int *bits, const uint32_t *mh, int F2, int K2,
                      uint64_t *klo, uint64_t *khi, cudaStream_t st);
geek_status group_tables(geek_ctx *ctx, Scratch &scr, int64_t n, int L, uint64_t *klo,
                         uint64_t *khi, int nbits, uint32_t *ids, int32_t *obj_bucket,
                         int64_t **boff_out, std::vector<int64_t> &nb, int64_t *NB_out,
                         cudaStream_t st);
int grid_for(int64_t work, int threads, int num_sms);

// Library-owned result of geek_hash.
struct geek_buckets {
    geek_ctx *ctx = nullptr;
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
};

struct silk_seeds {
    geek_ctx *ctx = nullptr;
    int64_t k = 0, n_ids = 0, n_multiset = 0;
    int64_t *off = nullptr;  // k + 1
    int32_t *ids = nullptr;  // n_ids
};

// silk.cu
geek_status silk_run(geek_ctx *ctx, const geek_buckets *b, const silk_params *p, silk_seeds *out,
                     cudaStream_t st);

// tc_assign.cu
geek_status assign_tc_bf16(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx, int64_t n, int d,
                           const double *centres, int64_t k, int32_t *labels, int32_t *flag_rows,
                           unsigned long long *n_flag, cudaStream_t st);

// assign.cu
geek_status assign_dense_centres(geek_ctx *ctx, Scratch &scr, const float *x, int64_t ldx,
                                 int64_t n, int d, const double *centres, int64_t k, int precision,
                                 int32_t *labels, geek_assign_stats *stats, cudaStream_t st);
geek_status centroids_from_seeds(geek_ctx *ctx, const float *x, int64_t ldx, int d,
                                 const silk_seeds *s, double *centres, cudaStream_t st);
geek_status assign_hetero(geek_ctx *ctx, Scratch &scr, const geek_buckets *b, const uint32_t *tok,
                          int n_cat, const silk_seeds *s, int32_t *labels, geek_assign_stats *stats,
                          cudaStream_t st);
geek_status assign_sets(geek_ctx *ctx, Scratch &scr, const int64_t *off, const uint32_t *items,
                        int64_t n, const silk_seeds *s, int32_t *labels, geek_assign_stats *stats,
                        cudaStream_t st);
