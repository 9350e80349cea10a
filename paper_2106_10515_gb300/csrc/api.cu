// C ABI: argument checking, staging and orchestration of the kernels in
// hash.cu / sort.cu / silk.cu / assign.cu.  Every entry point returns a
// geek_status and never lets an exception cross the ABI.
#include <new>

#include "internal.cuh"

// Result buffers are stream-ordered allocations on the call's stream (no
// device-wide synchronisation, so copies on other streams keep running).
geek_status own_alloc(geek_ctx *ctx, void **p, size_t bytes, cudaStream_t st) {
    if (alloc_injected_failure(ctx))
        return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed (injected)", bytes);
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed", bytes);
    }
    return GEEK_OK;
}

namespace {

cudaStream_t S(geek_stream s) { return (cudaStream_t)s; }

// Copies a host array to device scratch when the data set lives on the host.
template <class T>
geek_status stage(geek_ctx *ctx, Scratch &scr, const T *src, size_t count, bool host, const T **dst,
                  cudaStream_t st) {
    if (!host || src == nullptr) {
        *dst = src;
        return GEEK_OK;
    }
    T *d;
    GK_TRY(scr.alloc(&d, count));
    GK_CUDA(ctx, cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, st));
    *dst = d;
    return GEEK_OK;
}

void free_buckets(geek_buckets *b) {
    if (!b) return;
    for (void *p : {(void *)b->obj_bucket, (void *)b->boff, (void *)b->members, (void *)b->codes,
                    (void *)b->num_key, (void *)b->doph_tok})
        if (p) cudaFreeAsync(p, b->st);
    delete b;
}

geek_status check_data(geek_ctx *ctx, const geek_data *d) {
    if (!d) return set_error(ctx, GEEK_ERR_INVALID, "data is NULL");
    if (d->n < 0 || d->n > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_INVALID, "n out of range");
    if (d->mem != GEEK_MEM_DEVICE && d->mem != GEEK_MEM_HOST)
        return set_error(ctx, GEEK_ERR_INVALID, "bad mem");
    if (d->kind == GEEK_DENSE || d->kind == GEEK_HETERO) {
        if (d->d <= 0 || d->ldx < d->d || (d->n > 0 && !d->x))
            return set_error(ctx, GEEK_ERR_INVALID, "dense data needs x, d > 0 and ldx >= d");
    }
    if (d->kind == GEEK_HETERO && (d->n_cat <= 0 || (d->n > 0 && !d->cat)))
        return set_error(ctx, GEEK_ERR_INVALID, "hetero data needs cat tokens");
    if (d->kind == GEEK_SETS && (!d->set_off || (d->n > 0 && !d->set_items)))
        return set_error(ctx, GEEK_ERR_INVALID, "set data needs set_off and set_items");
    if (d->kind < 0 || d->kind > 2) return set_error(ctx, GEEK_ERR_INVALID, "bad kind");
    return GEEK_OK;
}

geek_status hash_impl(geek_ctx *ctx, const geek_data *data, const geek_hash_params *p,
                      geek_buckets **out, cudaStream_t st) {
    GK_TRY(check_data(ctx, data));
    if (!p || !out) return set_error(ctx, GEEK_ERR_INVALID, "params/out is NULL");
    *out = nullptr;
    const int kind = data->kind;
    const int64_t n = data->n;
    const int K = p->K, L = p->L;
    if (K <= 0 || L <= 0 || (int64_t)K * L > 4096) return set_error(ctx, GEEK_ERR_INVALID, "bad K/L");
    if (kind == GEEK_HETERO && p->Kc <= 0) return set_error(ctx, GEEK_ERR_INVALID, "hetero needs Kc > 0");
    if (kind != GEEK_HETERO && p->Kc != 0) return set_error(ctx, GEEK_ERR_INVALID, "Kc is for hetero data only");
    if (kind != GEEK_SETS) {
        if (!p->a || (p->proj == GEEK_PROJ_E2LSH && (!p->b || !(p->w > 0.0))))
            return set_error(ctx, GEEK_ERR_INVALID, "projection parameters missing");
        if (p->proj != GEEK_PROJ_E2LSH && p->proj != GEEK_PROJ_SRP && p->proj != GEEK_PROJ_QALSH)
            return set_error(ctx, GEEK_ERR_INVALID, "bad proj");
    }
    if (p->proj == GEEK_PROJ_QALSH && kind != GEEK_SETS) {
        if (kind != GEEK_DENSE || K != 1)
            return set_error(ctx, GEEK_ERR_INVALID, "QALSH (Alg. 1): dense data, K = 1, one table per projection");
        if (n > 0 && (p->t < 1 || p->t > n)) return set_error(ctx, GEEK_ERR_INVALID, "QALSH: need 1 <= t <= n");
    }
    if ((kind == GEEK_SETS || kind == GEEK_HETERO) && (!p->mh_a || !p->mh_b))
        return set_error(ctx, GEEK_ERR_INVALID, "MinHash coefficients missing");
    if (p->doph_bins != 0 && (kind != GEEK_SETS || p->doph_bins < 0 || p->doph_bins > 1024))
        return set_error(ctx, GEEK_ERR_INVALID, "DOPH: sets only, 1 <= bins <= 1024");
    if (p->precision != GEEK_PREC_FP32 && p->precision != GEEK_PREC_BF16X3)
        return set_error(ctx, GEEK_ERR_UNSUPPORTED, "projection precision other than FP32 or BF16X3");
    const bool host = data->mem == GEEK_MEM_HOST;

    Scratch scr(ctx, st);
    geek_buckets *b = new (std::nothrow) geek_buckets();
    if (!b) return set_error(ctx, GEEK_ERR_NOMEM, "host allocation");
    struct Guard {
        geek_buckets *b;
        ~Guard() { free_buckets(b); }
    } guard{b};
    b->ctx = ctx;
    b->st = st;
    b->kind = kind;
    b->n = n;
    b->L = L;
    b->K = K;
    b->Kc = p->Kc;

    const int F1 = kind == GEEK_SETS ? 0 : K * L;  // projection functions
    const int K1 = kind == GEEK_SETS ? 0 : K;
    const int K2 = kind == GEEK_SETS ? K : (kind == GEEK_HETERO ? p->Kc : 0);
    const int F2 = K2 * L;                         // MinHash functions
    b->F = kind == GEEK_SETS ? F2 : F1;

    int *fmin = nullptr, *fmax = nullptr, *bits = nullptr;
    const int Fm = std::max(1, F1);
    GK_TRY(scr.alloc(&fmin, Fm));
    GK_TRY(scr.alloc(&fmax, Fm));
    GK_TRY(scr.alloc(&bits, Fm));
    GK_TRY(own_alloc(ctx, (void **)&b->codes, sizeof(int32_t) * (size_t)n * std::max(1, b->F), st));

    if (kind == GEEK_DENSE && p->proj == GEEK_PROJ_QALSH) {  // Alg. 1
        const float *x;
        GK_TRY(stage(ctx, scr, data->x, (size_t)n * data->ldx, host, &x, st));
        GK_TRY(own_alloc(ctx, (void **)&b->members, sizeof(uint32_t) * (size_t)n * L, st));
        GK_TRY(own_alloc(ctx, (void **)&b->obj_bucket, sizeof(int32_t) * (size_t)n * L, st));
        GK_TRY(hash_qalsh(ctx, scr, x, data->ldx, n, data->d, p->a, L, p->t, b, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        guard.b = nullptr;
        *out = b;
        return GEEK_OK;
    }

    uint32_t *mh = nullptr;
    if (F1) {
        const float *x;
        GK_TRY(stage(ctx, scr, data->x, (size_t)n * data->ldx, host, &x, st));
        GK_TRY(project_dense(ctx, scr, x, data->ldx, n, data->d, p->a, p->b, F1, p->w,
                             p->proj == GEEK_PROJ_SRP, b->codes, fmin, fmax, &b->n_flagged,
                             &b->n_flagged_fp64, st, p->precision));
    }
    if (kind == GEEK_SETS) {
        const int64_t *off;
        int64_t n_items = 0;
        if (host) {
            n_items = data->set_off[n];
        } else {
            GK_CUDA(ctx, cudaMemcpyAsync(&n_items, data->set_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
        GK_TRY(stage(ctx, scr, data->set_off, (size_t)n + 1, host, &off, st));
        const uint32_t *items;
        GK_TRY(stage(ctx, scr, data->set_items, (size_t)n_items, host, &items, st));
        mh = (uint32_t *)b->codes;
        if (p->doph_bins > 0) {  // Alg. 3: DOPH reduction, then MinHash of the tokens
            // the reduced objects stay with the buckets: the assignment's
            // central vectors are modes over them (Sect. 3.3)
            uint64_t *tok;
            GK_TRY(own_alloc(ctx, (void **)&b->doph_tok, sizeof(uint64_t) * (size_t)std::max<int64_t>(n, 1) * p->doph_bins, st));
            tok = b->doph_tok;
            b->doph_bins = p->doph_bins;
            GK_TRY(doph_reduce(ctx, n, off, items, p->doph_bins, p->doph_a, p->doph_b, tok, st));
            GK_TRY(minhash_rows64(ctx, n, p->doph_bins, tok, F2, p->mh_a, p->mh_b, mh, st));
        } else {
            EvTimer tk(ctx, "kernel.minhash", st);
            tk.work = (double)n_items * F2;  // hash evaluations
            GK_TRY(minhash_rows(ctx, n, off, 0, items, F2, p->mh_a, p->mh_b, mh, st));
        }
    } else if (kind == GEEK_HETERO) {
        const uint32_t *tok;
        GK_TRY(stage(ctx, scr, data->cat, (size_t)n * data->n_cat, host, &tok, st));
        GK_TRY(scr.alloc(&mh, (size_t)n * F2));
        EvTimer tk(ctx, "kernel.minhash", st);
        tk.work = (double)n * data->n_cat * F2;  // hash evaluations
        GK_TRY(minhash_rows(ctx, n, nullptr, data->n_cat, tok, F2, p->mh_a, p->mh_b, mh, st));
    }
    std::vector<int> tbits;
    GK_TRY(key_layout(ctx, scr, fmin, fmax, L, K1, K2, bits, tbits, st));
    int nbits = 1;
    for (int v : tbits) nbits = std::max(nbits, v);
    b->key_bits_max = nbits;

    uint64_t *klo, *khi = nullptr;
    GK_TRY(scr.alloc(&klo, (size_t)n * L));
    if (nbits > 64) GK_TRY(scr.alloc(&khi, (size_t)n * L));
    GK_TRY(pack_keys(ctx, n, L, b->codes, F1, K1, fmin, bits, mh, F2, K2, klo, khi, st));

    if (kind == GEEK_HETERO) {
        // numeric-only key per table: the unified categorical attribute of
        // the numeric part (Sect. 3.3)
        std::vector<int> nbt;
        int nbn = 0;
        for (int l = 0; l < L; l++) nbn = std::max(nbn, tbits[l] - 32 * K2);
        if (nbn > 64) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "numeric key wider than 64 bits");
        GK_TRY(own_alloc(ctx, (void **)&b->num_key, sizeof(uint64_t) * (size_t)n * L, st));
        GK_TRY(pack_keys(ctx, n, L, b->codes, F1, K1, fmin, bits, nullptr, 0, 0, b->num_key, nullptr, st));
    }

    GK_TRY(own_alloc(ctx, (void **)&b->members, sizeof(uint32_t) * (size_t)n * L, st));
    GK_TRY(own_alloc(ctx, (void **)&b->obj_bucket, sizeof(int32_t) * (size_t)n * L, st));
    int64_t *boff = nullptr;
    GK_TRY(group_tables(ctx, scr, n, L, klo, khi, nbits, b->members, b->obj_bucket, &boff, b->nb, &b->NB, st));
    b->boff = boff;
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    guard.b = nullptr;
    *out = b;
    return GEEK_OK;
}

}  // namespace

unsigned long long g_geek_launches = 0;

extern "C" {

const char *geek_version(void) { return GEEK_VERSION_STRING; }

unsigned long long geek_launch_count(void) { return __atomic_load_n(&g_geek_launches, __ATOMIC_RELAXED); }

geek_status geek_timing_enable(geek_ctx *ctx, int on) {
    if (!ctx) return GEEK_ERR_INVALID;
    ctx->timing = on != 0;
    return GEEK_OK;
}

geek_status geek_timing_reset(geek_ctx *ctx) {
    if (!ctx) return GEEK_ERR_INVALID;
    ctx->resolve_timers();
    ctx->times.clear();
    return GEEK_OK;
}

geek_status geek_timing_get(const geek_ctx *ctx, const char *name, double *total_ms, int64_t *count,
                            double *total_work) {
    if (!ctx || !name) return GEEK_ERR_INVALID;
    ctx->resolve_timers();
    auto it = ctx->times.find(name);
    const bool f = it != ctx->times.end();
    if (total_ms) *total_ms = f ? it->second.ms : 0.0;
    if (count) *count = f ? it->second.count : 0;
    if (total_work) *total_work = f ? it->second.work : 0.0;
    return GEEK_OK;
}

geek_status geek_ctx_create(int device, geek_ctx **out) {
    if (!out) return GEEK_ERR_INVALID;
    *out = nullptr;
    geek_ctx *c = new (std::nothrow) geek_ctx();
    if (!c) return GEEK_ERR_NOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GEEK_ERR_CUDA;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    if (major * 10 + minor != 103) {
        delete c;
        return GEEK_ERR_UNSUPPORTED;  // built for sm_103a only
    }
    // keep freed stream-ordered memory cached in the device pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return GEEK_OK;
}

geek_status geek_ctx_destroy(geek_ctx *ctx) {
    delete ctx;
    return GEEK_OK;
}

geek_status geek_ctx_set_option(geek_ctx *ctx, int32_t option, int64_t value) {
    if (!ctx) return GEEK_ERR_INVALID;
    switch (option) {
    case GEEK_OPT_WAIT_LIMIT_NS:
        if (value < 1000 || value > 60000000000LL)
            return set_error(ctx, GEEK_ERR_INVALID, "wait limit %lld ns outside [1e3, 6e10]", (long long)value);
        ctx->lb_wait_ns = (unsigned long long)value;
        return GEEK_OK;
    case GEEK_OPT_TEST_STALL_TILE:
        if (value < -1 || value > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_INVALID, "bad stall tile");
        ctx->stall_tile = (int)value;
        return GEEK_OK;
    case GEEK_OPT_TEST_FAIL_ALLOC:
        if (value < -1) return set_error(ctx, GEEK_ERR_INVALID, "bad allocation countdown");
        ctx->fail_alloc_after = value;
        return GEEK_OK;
    default:
        return set_error(ctx, GEEK_ERR_INVALID, "unknown option %d", (int)option);
    }
}

const char *geek_last_error(const geek_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

geek_status geek_hash(geek_ctx *ctx, const geek_data *data, const geek_hash_params *p,
                      geek_buckets **out, geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        EvTimer tm(ctx, "hash", S(stream));
        return hash_impl(ctx, data, p, out, S(stream));
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_hash");
    }
}

geek_status geek_buckets_info_get(const geek_buckets *b, geek_buckets_info *info) {
    if (!b || !info) return GEEK_ERR_INVALID;
    info->n = b->n;
    info->L = b->L;
    info->key_bits_max = b->key_bits_max;
    info->n_buckets = b->NB;
    info->n_flagged = b->n_flagged;
    info->n_flagged_fp64 = b->n_flagged_fp64;
    return GEEK_OK;
}

geek_status geek_buckets_copy_out(const geek_buckets *b, int32_t *obj_bucket, int64_t *n_buckets,
                                  int64_t *bucket_off, int32_t *members, int32_t *codes,
                                  geek_stream stream) {
    if (!b) return GEEK_ERR_INVALID;
    geek_ctx *ctx = b->ctx;
    cudaStream_t st = S(stream);
    const size_t nl = (size_t)b->n * b->L;
    if (obj_bucket)
        GK_CUDA(ctx, cudaMemcpyAsync(obj_bucket, b->obj_bucket, nl * 4, cudaMemcpyDeviceToDevice, st));
    if (n_buckets)
        for (int l = 0; l < b->L; l++) n_buckets[l] = b->nb[l];
    if (bucket_off)
        GK_CUDA(ctx, cudaMemcpyAsync(bucket_off, b->boff, (b->NB + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if (members) GK_CUDA(ctx, cudaMemcpyAsync(members, b->members, nl * 4, cudaMemcpyDeviceToDevice, st));
    if (codes)
        GK_CUDA(ctx, cudaMemcpyAsync(codes, b->codes, (size_t)b->n * b->F * 4, cudaMemcpyDeviceToDevice, st));
    return GEEK_OK;
}

geek_status geek_buckets_free(geek_buckets *b) {
    free_buckets(b);
    return GEEK_OK;
}

geek_status silk_seed(geek_ctx *ctx, const geek_buckets *b, const silk_params *p, silk_seeds **out,
                      geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    if (!b || !p || !out) return set_error(ctx, GEEK_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (p->Ks < 1 || p->Ks > 4 || p->Ls < 1 || p->delta < 1 || !p->mh_a || !p->mh_b || !p->dd_a || !p->dd_b)
        return set_error(ctx, GEEK_ERR_INVALID, "bad SILK parameters");
    silk_seeds *s = new (std::nothrow) silk_seeds();
    if (!s) return set_error(ctx, GEEK_ERR_NOMEM, "host allocation");
    s->ctx = ctx;
    s->st = S(stream);
    geek_status st;
    try {
        EvTimer tm(ctx, "silk", S(stream));
        st = silk_run(ctx, b, p, s, S(stream));
    } catch (...) {
        st = set_error(ctx, GEEK_ERR_NOMEM, "host exception in silk_seed");
    }
    if (st != GEEK_OK) {
        silk_seeds_free(s);
        return st;
    }
    *out = s;
    return GEEK_OK;
}

geek_status silk_seeds_info(const silk_seeds *s, int64_t *k, int64_t *n_ids, int64_t *n_multiset) {
    if (!s) return GEEK_ERR_INVALID;
    if (k) *k = s->k;
    if (n_ids) *n_ids = s->n_ids;
    if (n_multiset) *n_multiset = s->n_multiset;
    return GEEK_OK;
}

geek_status silk_seeds_copy_out(const silk_seeds *s, int64_t *off, int32_t *ids, geek_stream stream) {
    if (!s) return GEEK_ERR_INVALID;
    geek_ctx *ctx = s->ctx;
    if (off) GK_CUDA(ctx, cudaMemcpyAsync(off, s->off, (s->k + 1) * 8, cudaMemcpyDeviceToDevice, S(stream)));
    if (ids && s->n_ids)
        GK_CUDA(ctx, cudaMemcpyAsync(ids, s->ids, s->n_ids * 4, cudaMemcpyDeviceToDevice, S(stream)));
    return GEEK_OK;
}

geek_status silk_seeds_free(silk_seeds *s) {
    if (!s) return GEEK_OK;
    if (s->off) cudaFreeAsync(s->off, s->st);
    if (s->ids) cudaFreeAsync(s->ids, s->st);
    delete s;
    return GEEK_OK;
}

struct geek_resident {
    void *buf[3] = {nullptr, nullptr, nullptr};  // x, set_off, set_items or cat
    size_t cap[3] = {0, 0, 0};                   // bytes
};

geek_status geek_resident_free(geek_resident *r) {
    if (!r) return GEEK_OK;
    for (void *p : r->buf) cudaFree(p);
    delete r;
    return GEEK_OK;
}

geek_status geek_data_upload(geek_ctx *ctx, const geek_data *host, geek_resident **res, geek_data *view,
                             geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        if (!res || !view) return set_error(ctx, GEEK_ERR_INVALID, "NULL argument");
        GK_TRY(check_data(ctx, host));
        if (host->mem != GEEK_MEM_HOST) return set_error(ctx, GEEK_ERR_INVALID, "upload needs host data");
        const int64_t n = host->n;
        size_t bytes[3] = {0, 0, 0};
        const void *src[3] = {nullptr, nullptr, nullptr};
        if (host->kind == GEEK_DENSE || host->kind == GEEK_HETERO) {
            bytes[0] = (size_t)n * host->ldx * sizeof(float);
            src[0] = host->x;
        }
        if (host->kind == GEEK_HETERO) {
            bytes[1] = (size_t)n * host->n_cat * sizeof(uint32_t);
            src[1] = host->cat;
        }
        if (host->kind == GEEK_SETS) {
            if (host->set_off[0] != 0 || host->set_off[n] < 0)
                return set_error(ctx, GEEK_ERR_INVALID, "set_off must start at 0 and ascend");
            bytes[1] = (size_t)(n + 1) * sizeof(int64_t);
            src[1] = host->set_off;
            bytes[2] = (size_t)host->set_off[n] * sizeof(uint32_t);
            src[2] = host->set_items;
        }
        geek_resident *r = *res ? *res : new (std::nothrow) geek_resident;
        if (!r) return set_error(ctx, GEEK_ERR_NOMEM, "host allocation");
        cudaStream_t st = S(stream);
        for (int j = 0; j < 3; ++j) {
            if (bytes[j] <= r->cap[j]) continue;
            void *p = nullptr;
            geek_status e = own_alloc(ctx, &p, bytes[j], st);
            if (e != GEEK_OK) {
                if (!*res) geek_resident_free(r);
                return e;
            }
            // the old buffer may still be read by work queued on `st`
            if (r->buf[j]) {
                cudaStreamSynchronize(st);
                cudaFree(r->buf[j]);
            }
            r->buf[j] = p;
            r->cap[j] = bytes[j];
        }
        for (int j = 0; j < 3; ++j)
            if (bytes[j]) {
                cudaError_t e = cudaMemcpyAsync(r->buf[j], src[j], bytes[j], cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) {
                    if (!*res) geek_resident_free(r);
                    cudaGetLastError();
                    return set_error(ctx, GEEK_ERR_CUDA, "upload copy: %s", cudaGetErrorString(e));
                }
            }
        *view = *host;
        view->mem = GEEK_MEM_DEVICE;
        view->x = host->kind == GEEK_SETS ? nullptr : (const float *)r->buf[0];
        view->cat = host->kind == GEEK_HETERO ? (const uint32_t *)r->buf[1] : nullptr;
        view->set_off = host->kind == GEEK_SETS ? (const int64_t *)r->buf[1] : nullptr;
        view->set_items = host->kind == GEEK_SETS ? (const uint32_t *)r->buf[2] : nullptr;
        *res = r;
        return GEEK_OK;
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_data_upload");
    }
}

geek_status geek_assign_centers(geek_ctx *ctx, const geek_data *data, const double *centers,
                                int64_t k, const geek_assign_params *p, int32_t *labels,
                                geek_assign_stats *stats, geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        GK_TRY(check_data(ctx, data));
        if (data->kind != GEEK_DENSE) return set_error(ctx, GEEK_ERR_INVALID, "dense data only");
        if (!p || !labels || (k > 0 && !centers) || k < 0 || k > 0x7FFFFFFFLL)
            return set_error(ctx, GEEK_ERR_INVALID, "bad assignment arguments");
        if (stats) *stats = geek_assign_stats{};
        cudaStream_t st = S(stream);
        EvTimer tm(ctx, "assign", st);
        Scratch scr(ctx, st);
        const bool host = data->mem == GEEK_MEM_HOST;
        const float *x;
        GK_TRY(stage(ctx, scr, data->x, (size_t)data->n * data->ldx, host, &x, st));
        int32_t *lab = labels;
        if (host) GK_TRY(scr.alloc(&lab, data->n));
        const double *c = centers;
        if (host && k) {
            double *dc;
            GK_TRY(scr.alloc(&dc, (size_t)k * data->d));
            GK_CUDA(ctx, cudaMemcpyAsync(dc, centers, sizeof(double) * k * data->d, cudaMemcpyHostToDevice, st));
            c = dc;
        }
        GK_TRY(assign_dense_centres(ctx, scr, x, data->ldx, data->n, data->d, c, k, p->precision, lab, stats, st));
        if (host) {
            GK_CUDA(ctx, cudaMemcpyAsync(labels, lab, sizeof(int32_t) * data->n, cudaMemcpyDeviceToHost, st));
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
        return GEEK_OK;
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_assign_centers");
    }
}

geek_status geek_cluster_radius(geek_ctx *ctx, const geek_data *data, const double *centers, int64_t k,
                                const int32_t *labels, double *radius, geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        GK_TRY(check_data(ctx, data));
        if (data->kind != GEEK_DENSE) return set_error(ctx, GEEK_ERR_INVALID, "dense data only");
        if (!labels || !radius || (k > 0 && !centers) || k < 0 || k > 0x7FFFFFFFLL)
            return set_error(ctx, GEEK_ERR_INVALID, "bad radius arguments");
        if (data->mem == GEEK_MEM_HOST) return set_error(ctx, GEEK_ERR_INVALID, "device data only");
        cudaStream_t st = S(stream);
        Scratch scr(ctx, st);
        return cluster_radius(ctx, scr, data->x, data->ldx, data->n, data->d, centers, k, labels, radius, st);
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_cluster_radius");
    }
}

geek_status geek_refine(geek_ctx *ctx, const geek_data *data, double *centers, int64_t k, int32_t passes,
                        const geek_assign_params *p, int32_t *labels, geek_assign_stats *stats,
                        geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        GK_TRY(check_data(ctx, data));
        if (data->kind != GEEK_DENSE || data->mem != GEEK_MEM_DEVICE)
            return set_error(ctx, GEEK_ERR_INVALID, "refine: dense device data only");
        if (!p || !labels || passes < 0 || k < 0 || k > 0x7FFFFFFFLL || (k > 0 && !centers))
            return set_error(ctx, GEEK_ERR_INVALID, "bad refine arguments");
        if (stats) *stats = geek_assign_stats{};
        cudaStream_t st = S(stream);
        EvTimer tm(ctx, "refine", st);
        Scratch scr(ctx, st);
        return refine_dense(ctx, scr, data->x, data->ldx, data->n, data->d, centers, k, passes, p->precision, labels,
                            stats, st);
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_refine");
    }
}

}  // extern "C"

namespace {

void free_centres(geek_centres *c) {
    if (!c) return;
    for (void *p : {(void *)c->centers, (void *)c->modes, (void *)c->item_off, (void *)c->items})
        if (p) cudaFreeAsync(p, c->st);
    delete c;
}

geek_status assign_impl(geek_ctx *ctx, const geek_data *data, const geek_buckets *b, const silk_seeds *s,
                        const geek_assign_params *p, int32_t *labels, double *centers, geek_assign_stats *stats,
                        geek_centres *keep, cudaStream_t st) {
    GK_TRY(check_data(ctx, data));
    if (!s || !p || !labels) return set_error(ctx, GEEK_ERR_INVALID, "NULL argument");
    if (stats) *stats = geek_assign_stats{};
    EvTimer tm(ctx, "assign", st);
    Scratch scr(ctx, st);
    const bool host = data->mem == GEEK_MEM_HOST;
    const int64_t n = data->n;
    int32_t *lab = labels;
    if (host) GK_TRY(scr.alloc(&lab, n));
    if (data->kind == GEEK_DENSE) {
        const float *x;
        GK_TRY(stage(ctx, scr, data->x, (size_t)n * data->ldx, host, &x, st));
        double *c = centers;
        if (!c || host) GK_TRY(scr.alloc(&c, (size_t)std::max<int64_t>(1, s->k) * data->d));
        GK_TRY(centroids_from_seeds(ctx, x, data->ldx, data->d, s, c, st));
        GK_TRY(assign_dense_centres(ctx, scr, x, data->ldx, n, data->d, c, s->k, p->precision, lab, stats, st));
        if (host && centers)
            GK_CUDA(ctx, cudaMemcpyAsync(centers, c, sizeof(double) * s->k * data->d, cudaMemcpyDeviceToHost, st));
        if (keep) {
            keep->kind = GEEK_DENSE;
            keep->k = s->k;
            keep->d = data->d;
            const size_t bytes = sizeof(double) * (size_t)s->k * data->d;
            GK_TRY(own_alloc(ctx, (void **)&keep->centers, bytes, st));
            if (bytes) GK_CUDA(ctx, cudaMemcpyAsync(keep->centers, c, bytes, cudaMemcpyDeviceToDevice, st));
        }
    } else if (data->kind == GEEK_HETERO) {
        if (!b || b->kind != GEEK_HETERO || b->n != n)
            return set_error(ctx, GEEK_ERR_INVALID, "hetero assignment needs its geek_buckets");
        const uint32_t *tok;
        GK_TRY(stage(ctx, scr, data->cat, (size_t)n * data->n_cat, host, &tok, st));
        GK_TRY(assign_hetero(ctx, scr, b, tok, data->n_cat, s, lab, stats, keep, st));
    } else {
        int64_t n_items = 0;
        if (host) {
            n_items = data->set_off[n];
        } else {
            GK_CUDA(ctx, cudaMemcpyAsync(&n_items, data->set_off + n, 8, cudaMemcpyDeviceToHost, st));
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
        if (b && b->kind == GEEK_SETS && b->doph_bins > 0) {
            if (b->n != n) return set_error(ctx, GEEK_ERR_INVALID, "buckets of another data set");
            GK_TRY(assign_doph(ctx, scr, b, s, lab, stats, keep, st));
        } else {
            const int64_t *off;
            const uint32_t *items;
            GK_TRY(stage(ctx, scr, data->set_off, (size_t)n + 1, host, &off, st));
            GK_TRY(stage(ctx, scr, data->set_items, (size_t)n_items, host, &items, st));
            GK_TRY(assign_sets(ctx, scr, off, items, n, s, lab, stats, keep, st));
        }
    }
    if (host) {
        GK_CUDA(ctx, cudaMemcpyAsync(labels, lab, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return GEEK_OK;
}

}  // namespace

extern "C" {

geek_status geek_assign(geek_ctx *ctx, const geek_data *data, const geek_buckets *b,
                        const silk_seeds *s, const geek_assign_params *p, int32_t *labels,
                        double *centers, geek_assign_stats *stats, geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    try {
        return assign_impl(ctx, data, b, s, p, labels, centers, stats, nullptr, S(stream));
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_assign");
    }
}

geek_status geek_assign_ex(geek_ctx *ctx, const geek_data *data, const geek_buckets *b, const silk_seeds *s,
                           const geek_assign_params *p, int32_t *labels, geek_assign_stats *stats,
                           geek_centres **centres, geek_stream stream) {
    if (!ctx) return GEEK_ERR_INVALID;
    if (!centres) return set_error(ctx, GEEK_ERR_INVALID, "NULL centres handle pointer");
    *centres = nullptr;
    geek_centres *c = new (std::nothrow) geek_centres();
    if (!c) return set_error(ctx, GEEK_ERR_NOMEM, "host allocation failed");
    c->ctx = ctx;
    c->st = S(stream);
    geek_status st;
    try {
        st = assign_impl(ctx, data, b, s, p, labels, nullptr, stats, c, S(stream));
    } catch (...) {
        st = set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_assign_ex");
    }
    if (st != GEEK_OK) {
        free_centres(c);
        return st;
    }
    *centres = c;
    return GEEK_OK;
}

geek_status geek_centres_info_get(const geek_centres *c, geek_centres_info *info) {
    if (!c || !info) return GEEK_ERR_INVALID;
    info->kind = c->kind;
    info->d = c->d;
    info->n_attr = c->n_attr;
    info->k = c->k;
    info->n_items = c->n_items;
    return GEEK_OK;
}

geek_status geek_centres_copy_out(const geek_centres *c, double *centers, int64_t *modes, int64_t *item_off,
                                  uint32_t *items, geek_stream stream) {
    if (!c) return GEEK_ERR_INVALID;
    geek_ctx *ctx = c->ctx;
    cudaStream_t st = S(stream);
    const auto D2D = cudaMemcpyDeviceToDevice;
    if (centers && c->centers && c->k * c->d)
        GK_CUDA(ctx, cudaMemcpyAsync(centers, c->centers, sizeof(double) * c->k * c->d, D2D, st));
    if (modes && c->modes && c->k * c->n_attr)
        GK_CUDA(ctx, cudaMemcpyAsync(modes, c->modes, sizeof(int64_t) * c->k * c->n_attr, D2D, st));
    if (item_off && c->item_off) GK_CUDA(ctx, cudaMemcpyAsync(item_off, c->item_off, sizeof(int64_t) * (c->k + 1), D2D, st));
    if (items && c->items && c->n_items)
        GK_CUDA(ctx, cudaMemcpyAsync(items, c->items, sizeof(uint32_t) * c->n_items, D2D, st));
    return GEEK_OK;
}

geek_status geek_centres_free(geek_centres *c) {
    free_centres(c);
    return GEEK_OK;
}

}  // extern "C"
