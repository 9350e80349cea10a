// Batched instances: the whole method (Sects. 3.1-3.3) for many independent
// dense data sets at once.
//
// The instances' objects are concatenated into one global row space
// (instance i owns rows [row_off[i], row_off[i + 1])), and every step runs
// once over all of them:
//  - hashing: one projection launch over every instance's row blocks, the
//    Dot2 / FP64 rechecks over one shared flag list, per-instance key layouts
//    (captured in a CUDA graph and replayed);
//  - grouping: one sort per table of (instance id | packed key), so buckets
//    never span instances and each instance keeps its lexicographic order;
//  - SILK: bins tagged by instance, each instance's own coefficients on its
//    local ids (silk_run with a SilkBatch);
//  - centroids, the persistent tcgen05 assignment over (instance, row tile)
//    units, the FP64 argmin decision and the statistics (captured in a
//    second CUDA graph, replayed while the seed counts are unchanged).
// The assignment's centre-tile width per instance comes from an autotuner
// that times the candidate widths on the batch's own data, once per
// (padded d, seed-count class) on a context.
#include <algorithm>
#include <new>

#include "internal.cuh"

namespace {

// seeds per instance: the instance of a seed is that of its first member
__global__ void k_seed_count(int64_t k, const int64_t *__restrict__ soff, const int32_t *__restrict__ sids,
                             const int64_t *__restrict__ row_off, int count, unsigned long long *__restrict__ kcnt) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k; s += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&kcnt[find_inst(row_off, count, (int64_t)sids[soff[s]])], 1ull);
}

// global member ids -> ids local to their instance
__global__ void k_local_ids(int64_t n, const int32_t *__restrict__ in, const int64_t *__restrict__ row_off, int count,
                            int32_t *__restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        out[p] = (int32_t)((int64_t)in[p] - row_off[find_inst(row_off, count, (int64_t)in[p])]);
}

// First bucket rank of every (instance, table): bucket g of table l (global
// index table_base[l] + r) starts its instance's range when it is the
// table's first bucket or its predecessor belongs to another instance.
__global__ void k_bucket_base(int64_t NB, const int64_t *__restrict__ table_base, int L,
                              const int64_t *__restrict__ boff, const uint32_t *__restrict__ members,
                              const int64_t *__restrict__ row_off, int count, int32_t *__restrict__ base) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < NB; g += (int64_t)gridDim.x * blockDim.x) {
        const int l = find_inst(table_base, L, g);
        const int64_t r = g - table_base[l];
        const int i = find_inst(row_off, count, (int64_t)members[boff[g]]);
        if (r == 0 || find_inst(row_off, count, (int64_t)members[boff[g - 1]]) != i) base[(int64_t)i * L + l] = (int32_t)r;
    }
}

__global__ void k_local_buckets(int64_t N, int L, const int32_t *__restrict__ ob, const int64_t *__restrict__ row_off,
                                int count, const int32_t *__restrict__ base, int32_t *__restrict__ out) {
    const int64_t tot = N * L;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / N);
        const int64_t r = e - (int64_t)l * N;
        out[e] = ob[e] - base[(int64_t)find_inst(row_off, count, r) * L + l];
    }
}

template <class T>
geek_status dalloc(geek_ctx *ctx, T **p, size_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, GEEK_ERR_NOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
    }
    return GEEK_OK;
}

template <class T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// seed-count class of the tile autotuner
int k_class(int64_t k) {
    int c = 0;
    for (int64_t lim = 64; c < 7 && k > lim; lim *= 2) c++;
    return c;
}

// default centre-tile width before (or without) tuning: the narrowest
// candidate that holds all centres, else the widest the mode allows
// (split-BF16 tiles need N * Kp <= 8192)
int tile_max(int d, int split) { return split ? (d <= 64 ? 128 : 64) : 256; }
int tile_default(int64_t k, int d, int split) {
    return std::min(tile_max(d, split), k <= 64 ? 64 : (k <= 128 ? 128 : 256));
}
// tuning-cache key: (padded d, seed-count class) under one precision setting
int class_key(int precision, int d, int64_t k) {
    return ((precision + 2) << 16) | ((d <= 64 ? 64 : 128) << 8) | k_class(k);
}

}  // namespace

struct geek_batch {
    geek_ctx *ctx = nullptr;
    int count = 0;
    geek_batch_params p{};
    std::vector<geek_instance> inst;
    std::vector<int64_t> row_off;  // host, count + 1
    int64_t N = 0;
    int F = 0, dmax = 0;
    cudaStream_t cs = nullptr;      // capture stream
    // ---- hash phase
    int32_t *codes = nullptr;
    ProjBatchBufs hb;
    std::vector<ProjArgs> P;
    cudaGraphExec_t g_hash = nullptr;
    int g_hash_kernels = 0;
    uint64_t *mh_a = nullptr, *mh_b = nullptr, *dd_a = nullptr, *dd_b = nullptr;  // stacked coefficients
    // ---- last run: buckets and seeds
    uint32_t *members = nullptr;
    int32_t *obj_bucket = nullptr;
    int64_t *boff = nullptr;
    std::vector<int64_t> nb;
    int64_t NB = 0;
    int key_bits = 0;
    int64_t n_flagged = 0, n_flagged_fp64 = 0;
    silk_seeds seeds;
    std::vector<int64_t> k;          // per instance
    std::vector<int64_t> seed_base;  // count + 1
    // ---- assignment phase (rebuilt when the seed counts change)
    bool a_ready = false;
    std::vector<int64_t> a_k;        // seed counts the phase was built for
    int32_t *a_labels = nullptr;     // labels pointer it was captured with
    TcPlan tc;
    std::vector<int> tile, split;    // per instance: centre-tile width, split-BF16 mode
    int64_t ktot = 0, ids_cap = 0, kd_tot = 0;
    int64_t *s_off = nullptr;        // seeds copied into plan-owned buffers
    int32_t *s_ids = nullptr;
    int64_t *seed_off_inst = nullptr;
    double *c64 = nullptr;
    float *c32 = nullptr, *cn32 = nullptr, *chi = nullptr, *clo = nullptr;
    unsigned *cmax_prep = nullptr;
    CenInst *cen = nullptr;
    CInst *cinst = nullptr;
    RInst *rinst = nullptr;
    SInst *sinst = nullptr;
    int2 *st_units = nullptr;
    int64_t n_st_units = 0;
    int64_t *st_uoff = nullptr;
    double *part_sum = nullptr, *sse_d = nullptr, *rmax_d = nullptr;
    float *part_max = nullptr;
    int32_t *flag_rows = nullptr;
    unsigned long long *n_flag = nullptr;
    DecideBufs dec;                  // grouping and FP32 / FP64 decision of flagged rows
    cudaGraphExec_t g_assign = nullptr;
    int g_assign_kernels = 0;
    std::vector<int64_t> cen_off;    // count + 1 (doubles)
    // ---- results of the last run
    std::vector<double> sse, rmax;
    int64_t n_recheck_rows = 0;
    int64_t n_fp64_rows = 0;
    int graph_launches = 0, graph_captures = 0, tuned = 0;

    void free_assign() {
        if (g_assign) cudaGraphExecDestroy(g_assign);
        g_assign = nullptr;
        tc_plan_free(&tc);
        dfree(s_off);
        dfree(s_ids);
        dfree(seed_off_inst);
        dfree(c64);
        dfree(c32);
        dfree(cn32);
        dfree(chi);
        dfree(clo);
        dfree(cmax_prep);
        dfree(cen);
        dfree(cinst);
        dfree(rinst);
        dfree(sinst);
        dfree(st_units);
        dfree(st_uoff);
        dfree(part_sum);
        dfree(part_max);
        dfree(sse_d);
        dfree(rmax_d);
        decide_bufs_free(dec);
        a_ready = false;
    }
    ~geek_batch() {
        free_assign();
        if (g_hash) cudaGraphExecDestroy(g_hash);
        dfree(codes);
        dfree(hb.P);
        dfree(hb.tile_off);
        dfree(hb.row_off);
        dfree(hb.anorm);
        dfree(hb.fmin);
        dfree(hb.fmax);
        dfree(hb.bits);
        dfree(hb.tbits);
        dfree(hb.flags);
        dfree(hb.flags2);
        dfree(hb.cnt);
        dfree(hb.cnt2);
        dfree(hb.status);
        dfree(mh_a);
        dfree(mh_b);
        dfree(dd_a);
        dfree(dd_b);
        dfree(members);
        dfree(obj_bucket);
        dfree(boff);
        dfree(seeds.off);
        dfree(seeds.ids);
        dfree(flag_rows);
        dfree(n_flag);
        if (cs) cudaStreamDestroy(cs);
    }
};

namespace {

geek_status batch_create(geek_ctx *ctx, const geek_instance *inst, int count, const geek_batch_params *p,
                         geek_batch *b) {
    if (!inst || !p || count < 1 || count > 65535) return set_error(ctx, GEEK_ERR_INVALID, "bad batch arguments");
    if (p->proj != GEEK_PROJ_E2LSH && p->proj != GEEK_PROJ_SRP) return set_error(ctx, GEEK_ERR_INVALID, "bad proj");
    if (p->K < 1 || p->L < 1 || p->K * p->L > 512)
        return set_error(ctx, p->K * p->L > 512 ? GEEK_ERR_UNSUPPORTED : GEEK_ERR_INVALID, "bad K/L");
    if (p->Ks < 1 || p->Ks > 4 || p->Ls < 1 || p->delta < 1) return set_error(ctx, GEEK_ERR_INVALID, "bad SILK parameters");
    if (p->tile_n != 0 && p->tile_n != 64 && p->tile_n != 128 && p->tile_n != 256)
        return set_error(ctx, GEEK_ERR_INVALID, "tile_n must be 0, 64, 128 or 256");
    if (p->precision != GEEK_PREC_AUTO && p->precision != GEEK_PREC_BF16 && p->precision != GEEK_PREC_BF16X3)
        return set_error(ctx, GEEK_ERR_INVALID, "batch precision must be GEEK_PREC_AUTO, BF16 or BF16X3");
    b->ctx = ctx;
    b->count = count;
    b->p = *p;
    b->inst.assign(inst, inst + count);
    b->F = p->K * p->L;
    b->row_off.assign(count + 1, 0);
    for (int i = 0; i < count; i++) {
        const geek_instance &I = inst[i];
        if (I.n < 0 || I.d < 1 || I.ldx < I.d || (I.n > 0 && !I.x) || !I.a || !I.mh_a || !I.mh_b || !I.dd_a ||
            !I.dd_b || (p->proj == GEEK_PROJ_E2LSH && (!I.b || !(I.w > 0.0))))
            return set_error(ctx, GEEK_ERR_INVALID, "instance %d: bad data or parameters", i);
        if (I.d > 128) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "instance %d: d > 128", i);
        b->row_off[i + 1] = b->row_off[i] + I.n;
        b->dmax = std::max(b->dmax, I.d);
    }
    b->N = b->row_off[count];
    if (b->N > 0x7FFFFFFFLL) return set_error(ctx, GEEK_ERR_UNSUPPORTED, "more than 2^31 - 1 objects in a batch");
    const int64_t N = b->N, F = b->F, L = p->L;
    GK_CUDA(ctx, cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
    GK_TRY(dalloc(ctx, &b->codes, (size_t)N * F));
    ProjBatchBufs &B = b->hb;
    GK_TRY(dalloc(ctx, &B.P, count));
    GK_TRY(dalloc(ctx, &B.tile_off, count + 1));
    GK_TRY(dalloc(ctx, &B.row_off, count + 1));
    GK_TRY(dalloc(ctx, &B.anorm, (size_t)count * F));
    GK_TRY(dalloc(ctx, &B.fmin, (size_t)count * F));
    GK_TRY(dalloc(ctx, &B.fmax, (size_t)count * F));
    GK_TRY(dalloc(ctx, &B.bits, (size_t)count * F));
    GK_TRY(dalloc(ctx, &B.tbits, (size_t)count * L));
    GK_TRY(dalloc(ctx, &B.cnt, 1));
    GK_TRY(dalloc(ctx, &B.cnt2, 1));
    GK_TRY(dalloc(ctx, &B.status, 1));
    B.cap = std::max<int64_t>(1 << 20, N * F / 16);
    GK_TRY(dalloc(ctx, &B.flags, B.cap));
    GK_TRY(dalloc(ctx, &B.flags2, B.cap));
    GK_CUDA(ctx, cudaMemcpy(B.row_off, b->row_off.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice));
    std::vector<DenseInst> di(count);
    for (int i = 0; i < count; i++)
        di[i] = DenseInst{inst[i].x, inst[i].ldx, inst[i].n, inst[i].d, inst[i].a, inst[i].b, inst[i].w};
    GK_TRY(proj_batch_setup(ctx, b->P, di, (int)F, p->proj == GEEK_PROJ_SRP, b->codes, b->row_off.data(), B));
    // SILK coefficients stacked instance-major
    const int64_t ms = (int64_t)p->Ls * p->Ks, ds = p->Ks;
    GK_TRY(dalloc(ctx, &b->mh_a, (size_t)count * ms));
    GK_TRY(dalloc(ctx, &b->mh_b, (size_t)count * ms));
    GK_TRY(dalloc(ctx, &b->dd_a, (size_t)count * ds));
    GK_TRY(dalloc(ctx, &b->dd_b, (size_t)count * ds));
    GK_TRY(dalloc(ctx, &b->members, (size_t)N * L));
    GK_TRY(dalloc(ctx, &b->obj_bucket, (size_t)N * L));
    GK_TRY(dalloc(ctx, &b->flag_rows, (size_t)std::max<int64_t>(N, 1)));
    GK_TRY(dalloc(ctx, &b->n_flag, 1));
    b->k.assign(count, 0);
    b->seed_base.assign(count + 1, 0);
    b->sse.assign(count, 0.0);
    b->rmax.assign(count, 0.0);
    b->tile.assign(count, 256);
    b->split.assign(count, 0);
    return GEEK_OK;
}

// Captures `enqueue(stream)` into a graph on the batch's capture stream;
// *kernels = its kernel nodes (the launch counter counts them per replay).
template <class Fn>
geek_status capture(geek_batch *b, cudaGraphExec_t *exec, int *kernels, Fn enqueue) {
    geek_ctx *ctx = b->ctx;
    cudaGraph_t g = nullptr;
    const unsigned long long before = geek_launch_count();
    GK_CUDA(ctx, cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    const geek_status rc = enqueue(b->cs);
    ctx->capturing = false;
    const cudaError_t e = cudaStreamEndCapture(b->cs, &g);
    __atomic_store_n(&g_geek_launches, before, __ATOMIC_RELAXED);  // nothing ran yet
    if (rc != GEEK_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return set_error(ctx, GEEK_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    *kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++*kernels;
    }
    const cudaError_t e2 = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return set_error(ctx, GEEK_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
    b->graph_captures++;
    return GEEK_OK;
}

geek_status launch(geek_batch *b, cudaGraphExec_t exec, int kernels, cudaStream_t st) {
    GK_CUDA(b->ctx, cudaGraphLaunch(exec, st));
    __atomic_fetch_add(&g_geek_launches, (unsigned long long)kernels, __ATOMIC_RELAXED);
    b->graph_launches++;
    return GEEK_OK;
}

}  // namespace

namespace {

// ---- hashing and grouping ---------------------------------------------------
geek_status run_hash(geek_batch *b, cudaStream_t st) {
    geek_ctx *ctx = b->ctx;
    const int count = b->count, F = b->F, L = b->p.L, K = b->p.K;
    const int srp = b->p.proj == GEEK_PROJ_SRP;
    for (int attempt = 0; attempt < 2; attempt++) {
        if (!b->g_hash)
            GK_TRY(capture(b, &b->g_hash, &b->g_hash_kernels, [&](cudaStream_t s) {
                return proj_batch_enqueue(ctx, b->P[0], count, F, L, K, srp, b->hb, s);
            }));
        {
            EvTimer tk(ctx, "batch.hash_graph", st);
            GK_TRY(launch(b, b->g_hash, b->g_hash_kernels, st));
        }
        unsigned long long c1 = 0, c2 = 0;
        int status = 0;
        GK_CUDA(ctx, cudaMemcpyAsync(&c1, b->hb.cnt, sizeof c1, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaMemcpyAsync(&c2, b->hb.cnt2, sizeof c2, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaMemcpyAsync(&status, b->hb.status, sizeof status, cudaMemcpyDeviceToHost, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        if ((int64_t)c1 > b->hb.cap) {
            // the shared flag list overflowed: grow it and capture again
            cudaGraphExecDestroy(b->g_hash);
            b->g_hash = nullptr;
            dfree(b->hb.flags);
            dfree(b->hb.flags2);
            b->hb.cap = (int64_t)c1;
            GK_TRY(dalloc(ctx, &b->hb.flags, b->hb.cap));
            GK_TRY(dalloc(ctx, &b->hb.flags2, b->hb.cap));
            for (auto &A : b->P) {
                A.flags = b->hb.flags;
                A.flag_cap = b->hb.cap;
            }
            GK_CUDA(ctx, cudaMemcpy(b->hb.P, b->P.data(), sizeof(ProjArgs) * count, cudaMemcpyHostToDevice));
            continue;
        }
        if (status == GEEK_ERR_OVERFLOW) return set_error(ctx, GEEK_ERR_OVERFLOW, "E2LSH code outside int32 or key too wide");
        if (status) return set_error(ctx, (geek_status)status, "batched hashing failed");
        b->n_flagged = (int64_t)c1;
        b->n_flagged_fp64 = (int64_t)c2;
        break;
    }
    if (!b->g_hash) return set_error(ctx, GEEK_ERR_CUDA, "projection flag list did not converge");
    // composite key: instance id above the widest per-instance key
    std::vector<int> tbits((size_t)count * L);
    GK_CUDA(ctx, cudaMemcpy(tbits.data(), b->hb.tbits, sizeof(int) * tbits.size(), cudaMemcpyDeviceToHost));
    int B = 0;
    for (int v : tbits) B = std::max(B, v);
    const int ib = bit_length_u64((uint64_t)(count - 1));
    const int nbits = std::max(1, B + ib);
    if (nbits > 128) return set_error(ctx, GEEK_ERR_OVERFLOW, "instance id + table key wider than 128 bits");
    b->key_bits = nbits;
    EvTimer tg(ctx, "batch.group", st);
    Scratch scr(ctx, st);
    const int64_t N = b->N;
    uint64_t *klo, *khi = nullptr;
    GK_TRY(scr.alloc(&klo, (size_t)N * L));
    if (nbits > 64) GK_TRY(scr.alloc(&khi, (size_t)N * L));
    GK_TRY(pack_keys_batch(ctx, N, L, b->codes, K, b->hb.row_off, count, b->hb.fmin, b->hb.bits, B, klo, khi, st));
    dfree(b->boff);
    GK_TRY(group_tables(ctx, scr, N, L, klo, khi, nbits, b->members, b->obj_bucket, &b->boff, b->nb, &b->NB, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    return GEEK_OK;
}

// ---- SILK and the per-instance seed ranges ----------------------------------
geek_status run_silk(geek_batch *b, cudaStream_t st) {
    geek_ctx *ctx = b->ctx;
    const int count = b->count;
    geek_buckets gb;
    gb.ctx = ctx;
    gb.kind = GEEK_DENSE;
    gb.n = b->N;
    gb.L = b->p.L;
    gb.K = b->p.K;
    gb.F = b->F;
    gb.NB = b->NB;
    gb.nb = b->nb;
    gb.obj_bucket = b->obj_bucket;
    gb.boff = b->boff;
    gb.members = b->members;
    silk_params sp{b->p.Ks, b->p.Ls, b->p.delta, b->mh_a, b->mh_b, b->dd_a, b->dd_b};
    SilkBatch sb;
    sb.row_off = b->hb.row_off;
    sb.count = count;
    dfree(b->seeds.off);
    dfree(b->seeds.ids);
    b->seeds = silk_seeds();
    b->seeds.ctx = ctx;
    geek_status rc;
    {
        EvTimer tk(ctx, "batch.silk", st);
        rc = silk_run(ctx, &gb, &sp, &b->seeds, st, &sb);
    }
    // the view does not own the bucket arrays
    gb.obj_bucket = nullptr;
    gb.boff = nullptr;
    gb.members = nullptr;
    GK_TRY(rc);
    Scratch scr(ctx, st);
    unsigned long long *kc;
    GK_TRY(scr.alloc(&kc, count));
    GK_CUDA(ctx, cudaMemsetAsync(kc, 0, sizeof(unsigned long long) * count, st));
    if (b->seeds.k > 0) {
        GK_COUNT();
        k_seed_count<<<grid_for(b->seeds.k, 256, ctx->num_sms), 256, 0, st>>>(b->seeds.k, b->seeds.off, b->seeds.ids,
                                                                            b->hb.row_off, count, kc);
        GK_LAUNCH(ctx);
    }
    std::vector<unsigned long long> h(count);
    GK_CUDA(ctx, cudaMemcpyAsync(h.data(), kc, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    for (int i = 0; i < count; i++) {
        b->k[i] = (int64_t)h[i];
        b->seed_base[i + 1] = b->seed_base[i] + b->k[i];
    }
    return GEEK_OK;
}

}  // namespace

namespace {

// ---- assignment phase ---------------------------------------------------------
// Buffers and descriptors for the current seed counts b->k and labels.
geek_status build_assign(geek_batch *b, int32_t *labels, cudaStream_t st) {
    geek_ctx *ctx = b->ctx;
    const int count = b->count;
    b->free_assign();
    b->ktot = b->seed_base[count];
    b->ids_cap = std::max<int64_t>(b->seeds.n_ids, 1);
    b->cen_off.assign(count + 1, 0);
    for (int i = 0; i < count; i++) b->cen_off[i + 1] = b->cen_off[i] + b->k[i] * b->inst[i].d;
    b->kd_tot = b->cen_off[count];
    const int64_t kt = std::max<int64_t>(b->ktot, 1), kd = std::max<int64_t>(b->kd_tot, 1);
    GK_TRY(dalloc(ctx, &b->s_off, kt + 1));
    GK_TRY(dalloc(ctx, &b->s_ids, b->ids_cap));
    GK_TRY(dalloc(ctx, &b->seed_off_inst, count + 1));
    GK_TRY(dalloc(ctx, &b->c64, kd));
    GK_TRY(dalloc(ctx, &b->c32, kd));
    GK_TRY(dalloc(ctx, &b->chi, kd));
    GK_TRY(dalloc(ctx, &b->clo, kd));
    GK_TRY(dalloc(ctx, &b->cn32, kt));
    GK_TRY(dalloc(ctx, &b->cmax_prep, count));
    GK_TRY(dalloc(ctx, &b->cen, count));
    GK_TRY(dalloc(ctx, &b->cinst, count));
    GK_TRY(dalloc(ctx, &b->rinst, count));
    GK_TRY(dalloc(ctx, &b->sinst, count));
    GK_TRY(dalloc(ctx, &b->sse_d, count));
    GK_TRY(dalloc(ctx, &b->rmax_d, count));
    GK_TRY(dalloc(ctx, &b->st_uoff, count + 1));
    std::vector<CenInst> cen(count);
    std::vector<CInst> ci(count);
    std::vector<RInst> ri(count);
    std::vector<SInst> si(count);
    std::vector<int2> su;
    std::vector<int64_t> suoff(count + 1, 0);
    std::vector<TcPlanInst> tp(count);
    for (int i = 0; i < count; i++) {
        const geek_instance &I = b->inst[i];
        const int64_t r0 = b->row_off[i];
        double *c = b->c64 + b->cen_off[i];
        float *c32 = b->c32 + b->cen_off[i];
        cen[i] = CenInst{I.x, I.ldx, I.d, r0, b->seed_base[i], c};
        ci[i] = CInst{c, c32, b->cn32 + b->seed_base[i], b->cmax_prep + i, I.d, b->seed_base[i]};
        ri[i] = RInst{I.x, I.ldx, I.d, c32, b->cn32 + b->seed_base[i], c, b->k[i], b->cmax_prep + i, labels + r0, r0};
        si[i] = SInst{I.x, I.ldx, I.n, I.d, b->chi + b->cen_off[i], b->clo + b->cen_off[i], b->k[i], labels + r0};
        for (int64_t r = 0; r < ceil_div(I.n, 128); r++) su.push_back(make_int2(i, (int)r));
        suoff[i + 1] = (int64_t)su.size();
        // mode and tile: forced, tuned earlier on this context, or defaults
        int split = b->p.precision == GEEK_PREC_BF16X3 || b->p.precision == GEEK_PREC_AUTO;
        int N = tile_default(b->k[i], I.d, split);
        auto it = ctx->tile_cache.find(class_key(b->p.precision, I.d, b->k[i]));
        if (it != ctx->tile_cache.end() && !b->p.tile_n) {
            N = it->second & 0xFFFF;
            split = it->second >> 16;
        }
        if (b->p.tile_n) N = std::min(b->p.tile_n, tile_max(I.d, split));
        b->tile[i] = N;
        b->split[i] = split;
        tp[i] = TcPlanInst{I.x, I.ldx, I.n, I.d, c, b->k[i], labels + r0, r0, N, split};
    }
    b->n_st_units = (int64_t)su.size();
    GK_TRY(dalloc(ctx, &b->st_units, std::max<int64_t>(b->n_st_units, 1)));
    GK_TRY(dalloc(ctx, &b->part_sum, std::max<int64_t>(b->n_st_units, 1)));
    GK_TRY(dalloc(ctx, &b->part_max, std::max<int64_t>(b->n_st_units, 1)));
    GK_CUDA(ctx, cudaMemcpy(b->seed_off_inst, b->seed_base.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(b->cen, cen.data(), sizeof(CenInst) * count, cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(b->cinst, ci.data(), sizeof(CInst) * count, cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(b->rinst, ri.data(), sizeof(RInst) * count, cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(b->sinst, si.data(), sizeof(SInst) * count, cudaMemcpyHostToDevice));
    GK_CUDA(ctx, cudaMemcpy(b->st_uoff, suoff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice));
    if (!su.empty()) GK_CUDA(ctx, cudaMemcpy(b->st_units, su.data(), sizeof(int2) * su.size(), cudaMemcpyHostToDevice));
    b->tc.allow_split = b->p.precision == GEEK_PREC_AUTO;
    GK_TRY(tc_plan_build(ctx, nullptr, tp, &b->tc, st));
    GK_TRY(decide_bufs_alloc(ctx, nullptr, count, b->N, b->dec));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    b->a_k = b->k;
    b->a_labels = labels;
    b->a_ready = true;
    return GEEK_OK;
}

// centroids, centre preparation and the BF16 conversions (no host sync)
geek_status enqueue_centres(geek_batch *b, cudaStream_t s) {
    geek_ctx *ctx = b->ctx;
    GK_TRY(centroids_batch(ctx, b->cen, b->seed_off_inst, b->count, b->ktot, b->dmax, b->s_off, b->s_ids, s));
    GK_CUDA(ctx, cudaMemsetAsync(b->cmax_prep, 0, sizeof(unsigned) * b->count, s));
    GK_TRY(centre_prep_batch(ctx, b->cinst, b->seed_off_inst, b->count, b->ktot, s));
    GK_TRY(tc_plan_convert(ctx, b->tc, s));
    return GEEK_OK;
}

// the whole assignment phase (no host sync, no allocation: captured)
geek_status enqueue_assign(geek_batch *b, int32_t *labels, cudaStream_t s) {
    geek_ctx *ctx = b->ctx;
    GK_CUDA(ctx, cudaMemsetAsync(b->n_flag, 0, sizeof(unsigned long long), s));
    GK_TRY(fill_labels(ctx, labels, b->N, -1, s));
    GK_TRY(enqueue_centres(b, s));
    GK_TRY(tc_plan_launch(ctx, b->tc, b->flag_rows, b->n_flag, s));
    GK_TRY(decide_flags(ctx, b->rinst, b->hb.row_off, b->count, b->dmax, b->flag_rows, b->n_flag, b->dec, s));
    GK_TRY(centre_split(ctx, b->c64, b->kd_tot, b->chi, b->clo, s));
    GK_TRY(stats_batch(ctx, b->sinst, b->st_units, b->n_st_units, b->st_uoff, b->count, b->part_sum, b->part_max,
                       b->sse_d, b->rmax_d, s));
    return GEEK_OK;
}

// Chooses, for every (padded d, seed-count class) of the batch that the
// context has not tuned yet, the assignment mode (BF16 or split-BF16) and the
// centre-tile width by timing each candidate on that class's own instances:
// the tcgen05 pass plus the FP64 decision of the rows it leaves uncertain
// (a wide BF16 window trades tensor work for rechecks).  The choice is
// recorded on the context.
geek_status autotune(geek_batch *b, cudaStream_t st) {
    geek_ctx *ctx = b->ctx;
    std::map<int, std::vector<int>> classes;
    for (int i = 0; i < b->count; i++) {
        if (b->inst[i].n == 0 || b->k[i] == 0) continue;
        const int key = class_key(b->p.precision, b->inst[i].d, b->k[i]);
        if (!ctx->tile_cache.count(key)) classes[key].push_back(i);
    }
    if (classes.empty()) return GEEK_OK;
    EvTimer tk(ctx, "batch.autotune", st);
    GK_TRY(enqueue_centres(b, st));  // centroids, centre preparation and conversions
    std::vector<int> modes;
    if (b->p.precision != GEEK_PREC_BF16X3) modes.push_back(0);
    if (b->p.precision != GEEK_PREC_BF16) modes.push_back(1);
    const int *cand;
    const int nc = tc_tile_candidates(&cand);
    std::map<int, std::pair<float, int>> best;  // class -> (ms, N | split << 16)
    cudaEvent_t e0, e1;
    GK_CUDA(ctx, cudaEventCreate(&e0));
    GK_CUDA(ctx, cudaEventCreate(&e1));
    geek_status rc = GEEK_OK;
    std::vector<int> N = b->tile, split = b->split;
    for (int mode : modes) {
        for (auto &c : classes)
            for (int i : c.second) {
                split[i] = mode;
                N[i] = tile_default(b->k[i], b->inst[i].d, mode);
            }
        rc = tc_plan_set_modes(ctx, &b->tc, N, split, st);
        if (rc == GEEK_OK) rc = tc_plan_convert(ctx, b->tc, st);
        for (auto c = classes.begin(); c != classes.end() && rc == GEEK_OK; ++c) {
            // at most ~8 units per SM of this class's instances
            std::vector<int> which;
            int64_t units = 0;
            for (int i : c->second) {
                if (units > (int64_t)ctx->num_sms * 8) break;
                which.push_back(i);
                units += ceil_div(b->inst[i].n, 128);
            }
            const int dcls = b->inst[c->second[0]].d;
            for (int q = 0; q < nc && rc == GEEK_OK; q++) {
                if (cand[q] > tile_max(dcls, mode) || (b->p.tile_n && cand[q] != std::min(b->p.tile_n, tile_max(dcls, mode))))
                    continue;
                for (int i : c->second) N[i] = cand[q];
                rc = tc_plan_set_modes(ctx, &b->tc, N, split, st);
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && rc == GEEK_OK; rep++) {
                    cudaMemsetAsync(b->n_flag, 0, sizeof(unsigned long long), st);
                    cudaEventRecord(e0, st);
                    rc = tc_plan_launch_subset(ctx, &b->tc, which, b->flag_rows, b->n_flag, st);
                    if (rc == GEEK_OK)
                        rc = decide_flags(ctx, b->rinst, b->hb.row_off, b->count, b->dmax, b->flag_rows, b->n_flag,
                                          b->dec, st);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess && rc == GEEK_OK)
                        rc = set_error(ctx, GEEK_ERR_CUDA, "autotune run failed: %s", cudaGetErrorString(cudaGetLastError()));
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = std::min(ms, t);
                }
                if (rc == GEEK_OK) rc = tc_plan_check(ctx, b->tc, st);
                auto &bb = best[c->first];
                if (rc == GEEK_OK && (bb.second == 0 || ms < bb.first)) bb = {ms, cand[q] | (mode << 16)};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GK_TRY(rc);
    for (auto &c : classes) {
        const int v = best[c.first].second;
        ctx->tile_cache[c.first] = v;
        for (int i : c.second) {
            N[i] = v & 0xFFFF;
            split[i] = v >> 16;
        }
        b->tuned++;
    }
    b->tile = N;
    b->split = split;
    GK_TRY(tc_plan_set_modes(ctx, &b->tc, N, split, st));
    GK_CUDA(ctx, cudaStreamSynchronize(st));
    return GEEK_OK;
}

geek_status run_assign(geek_batch *b, int32_t *labels, cudaStream_t st) {
    geek_ctx *ctx = b->ctx;
    const int count = b->count;
    const bool rebuild = !b->a_ready || b->a_k != b->k || b->a_labels != labels || b->seeds.n_ids > b->ids_cap;
    if (rebuild) GK_TRY(build_assign(b, labels, st));
    // this run's seeds into the plan-owned buffers the graph reads
    GK_CUDA(ctx, cudaMemcpyAsync(b->s_off, b->seeds.off, sizeof(int64_t) * (b->ktot + 1), cudaMemcpyDeviceToDevice, st));
    if (b->seeds.n_ids)
        GK_CUDA(ctx, cudaMemcpyAsync(b->s_ids, b->seeds.ids, sizeof(int32_t) * b->seeds.n_ids, cudaMemcpyDeviceToDevice, st));
    if (rebuild && (!b->p.tile_n || b->p.precision == GEEK_PREC_AUTO)) GK_TRY(autotune(b, st));
    if (!b->g_assign)
        GK_TRY(capture(b, &b->g_assign, &b->g_assign_kernels, [&](cudaStream_t s) { return enqueue_assign(b, labels, s); }));
    {
        EvTimer tk(ctx, "batch.assign_graph", st);
        GK_TRY(launch(b, b->g_assign, b->g_assign_kernels, st));
    }
    unsigned long long nf = 0, nf64 = 0;
    GK_CUDA(ctx, cudaMemcpyAsync(&nf, b->n_flag, sizeof nf, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaMemcpyAsync(&nf64, b->dec.n_flag2, sizeof nf64, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaMemcpyAsync(b->sse.data(), b->sse_d, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
    GK_CUDA(ctx, cudaMemcpyAsync(b->rmax.data(), b->rmax_d, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
    GK_TRY(tc_plan_check(ctx, b->tc, st));  // synchronises
    b->n_recheck_rows = (int64_t)nf;
    b->n_fp64_rows = (int64_t)nf64;
    return GEEK_OK;
}

}  // namespace

extern "C" {

geek_status geek_batch_create(geek_ctx *ctx, const geek_instance *inst, int32_t count, const geek_batch_params *p,
                              geek_batch **out) {
    if (!ctx) return GEEK_ERR_INVALID;
    if (!out) return set_error(ctx, GEEK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    geek_batch *b = new (std::nothrow) geek_batch();
    if (!b) return set_error(ctx, GEEK_ERR_NOMEM, "host allocation");
    geek_status rc;
    try {
        rc = batch_create(ctx, inst, count, p, b);
        if (rc == GEEK_OK) {
            // stack the SILK coefficients instance-major
            const int64_t ms = (int64_t)p->Ls * p->Ks, ds = p->Ks;
            for (int i = 0; i < count && rc == GEEK_OK; i++) {
                if (cudaMemcpy(b->mh_a + i * ms, inst[i].mh_a, 8 * ms, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                    cudaMemcpy(b->mh_b + i * ms, inst[i].mh_b, 8 * ms, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                    cudaMemcpy(b->dd_a + i * ds, inst[i].dd_a, 8 * ds, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                    cudaMemcpy(b->dd_b + i * ds, inst[i].dd_b, 8 * ds, cudaMemcpyDeviceToDevice) != cudaSuccess)
                    rc = set_error(ctx, GEEK_ERR_CUDA, "copy of SILK coefficients failed: %s",
                                   cudaGetErrorString(cudaGetLastError()));
            }
        }
    } catch (...) {
        rc = set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_batch_create");
    }
    if (rc != GEEK_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return GEEK_OK;
}

geek_status geek_batch_run(geek_batch *b, int32_t *labels, geek_stream stream) {
    if (!b) return GEEK_ERR_INVALID;
    geek_ctx *ctx = b->ctx;
    if (!labels && b->N > 0) return set_error(ctx, GEEK_ERR_INVALID, "labels is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        EvTimer tm(ctx, "batch", st);
        GK_TRY(run_hash(b, st));
        GK_TRY(run_silk(b, st));
        GK_TRY(run_assign(b, labels, st));
        return GEEK_OK;
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_batch_run");
    }
}

geek_status geek_batch_info_get(const geek_batch *b, geek_batch_info *info) {
    if (!b || !info) return GEEK_ERR_INVALID;
    info->count = b->count;
    info->n_total = b->N;
    info->k_total = b->seed_base[b->count];
    info->n_buckets = b->NB;
    info->n_flagged = b->n_flagged;
    info->n_flagged_fp64 = b->n_flagged_fp64;
    info->n_recheck_rows = b->n_recheck_rows;
    info->n_fp64_rows = b->n_fp64_rows;
    info->key_bits = b->key_bits;
    info->graph_launches = b->graph_launches;
    info->graph_captures = b->graph_captures;
    info->tuned_classes = b->tuned;
    return GEEK_OK;
}

geek_status geek_batch_instance_stats(const geek_batch *b, int64_t *k, double *sse, double *radius_max,
                                      int32_t *tile_n, int32_t *precision) {
    if (!b) return GEEK_ERR_INVALID;
    for (int i = 0; i < b->count; i++) {
        if (k) k[i] = b->k[i];
        if (sse) sse[i] = b->sse[i];
        if (radius_max) radius_max[i] = b->rmax[i];
        if (tile_n) tile_n[i] = b->tile[i];
        if (precision) precision[i] = b->split[i] ? GEEK_PREC_BF16X3 : GEEK_PREC_BF16;
    }
    return GEEK_OK;
}

geek_status geek_batch_seed_ids_count(const geek_batch *b, int64_t *n_ids) {
    if (!b || !n_ids) return GEEK_ERR_INVALID;
    *n_ids = b->seeds.n_ids;
    return GEEK_OK;
}

geek_status geek_batch_copy_out(const geek_batch *b, int32_t *codes, int32_t *obj_bucket, int64_t *seed_off,
                                int32_t *seed_ids, double *centres, geek_stream stream) {
    if (!b) return GEEK_ERR_INVALID;
    geek_ctx *ctx = b->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    const int count = b->count, L = b->p.L;
    const int64_t N = b->N;
    try {
        if (codes && N) GK_CUDA(ctx, cudaMemcpyAsync(codes, b->codes, sizeof(int32_t) * N * b->F, cudaMemcpyDeviceToDevice, st));
        if (obj_bucket && N) {
            Scratch scr(ctx, st);
            int32_t *base;
            int64_t *tb;
            GK_TRY(scr.alloc(&base, (size_t)count * L));
            GK_TRY(scr.alloc(&tb, L + 1));
            std::vector<int64_t> h(L + 1, 0);
            for (int l = 0; l < L; l++) h[l + 1] = h[l] + b->nb[l];
            GK_CUDA(ctx, cudaMemcpyAsync(tb, h.data(), sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice, st));
            GK_CUDA(ctx, cudaMemsetAsync(base, 0, sizeof(int32_t) * count * L, st));
            GK_COUNT();
            k_bucket_base<<<grid_for(b->NB, 256, ctx->num_sms), 256, 0, st>>>(b->NB, tb, L, b->boff, b->members,
                                                                            b->hb.row_off, count, base);
            GK_COUNT();
            k_local_buckets<<<grid_for(N * L, 256, ctx->num_sms), 256, 0, st>>>(N, L, b->obj_bucket, b->hb.row_off,
                                                                              count, base, obj_bucket);
            GK_LAUNCH(ctx);
            GK_CUDA(ctx, cudaStreamSynchronize(st));
        }
        const int64_t kt = b->seed_base[count];
        if (seed_off)
            GK_CUDA(ctx, cudaMemcpyAsync(seed_off, b->seeds.off, sizeof(int64_t) * (kt + 1), cudaMemcpyDeviceToDevice, st));
        if (seed_ids && b->seeds.n_ids) {
            GK_COUNT();
            k_local_ids<<<grid_for(b->seeds.n_ids, 256, ctx->num_sms), 256, 0, st>>>(b->seeds.n_ids, b->seeds.ids,
                                                                                   b->hb.row_off, count, seed_ids);
            GK_LAUNCH(ctx);
        }
        if (centres && b->a_ready && b->kd_tot)
            GK_CUDA(ctx, cudaMemcpyAsync(centres, b->c64, sizeof(double) * b->kd_tot, cudaMemcpyDeviceToDevice, st));
        GK_CUDA(ctx, cudaStreamSynchronize(st));
        return GEEK_OK;
    } catch (...) {
        return set_error(ctx, GEEK_ERR_NOMEM, "host exception in geek_batch_copy_out");
    }
}

geek_status geek_batch_destroy(geek_batch *b) {
    delete b;
    return GEEK_OK;
}

}  // extern "C"
