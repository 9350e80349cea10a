/*
 * geek.h - C ABI of the GB300 GEEK library: bucketing (data transformation),
 * SILK seeding and one-pass assignment, after Luo, Huang and Tung, "A Generic
 * Distributed Clustering Framework for Massive Data" (Sect. 3).
 *
 * Conventions
 *  - Every array argument is DEVICE memory owned by the caller unless the
 *    comment says otherwise; the library never frees caller memory.
 *  - Work is enqueued on the caller's CUDA stream (geek_stream is a
 *    cudaStream_t; NULL selects the legacy default stream).  Calls whose
 *    output size depends on the data (geek_hash, silk_seed) read a few counts
 *    back to the host and therefore return only after those counts are known;
 *    the bulk outputs they own stay stream-ordered.
 *  - Outputs whose size depends on the data live in opaque library-owned
 *    handles (geek_buckets, silk_seeds): *_info gives sizes, *_copy_out
 *    copies into caller buffers, *_free releases the handle.
 *  - Random parameters of the method (E2LSH projections, MinHash and SILK
 *    hash coefficients) are inputs; the library draws nothing.  No call takes
 *    a number of clusters k: SILK decides it (Sect. 3.2).
 *  - Every call returns a geek_status.  Nothing aborts or throws across the
 *    ABI; geek_last_error() describes the last failure on a context.
 *  - Results are deterministic and bit-exact against an FP64 reference
 *    definition (see each call): fast single-precision or tensor-core paths
 *    recompute in FP64 every element whose rounding-error window could change
 *    an integer outcome (a bucket code, a sign, an argmin).
 */
#ifndef GEEK_H
#define GEEK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum geek_status {
    GEEK_OK = 0,
    GEEK_ERR_INVALID = 1,     /* bad argument, shape or pointer */
    GEEK_ERR_NOMEM = 2,       /* device or host allocation failed */
    GEEK_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed */
    GEEK_ERR_TIMEOUT = 4,     /* a bounded device wait expired */
    GEEK_ERR_OVERFLOW = 5,    /* a code or key does not fit its field */
    GEEK_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} geek_status;

typedef struct geek_ctx geek_ctx;
typedef struct geek_buckets geek_buckets;
typedef struct silk_seeds silk_seeds;
typedef void *geek_stream; /* cudaStream_t */

/* data kinds (Sect. 2.1 problem settings) */
enum { GEEK_DENSE = 0, GEEK_SETS = 1, GEEK_HETERO = 2 };
/* where the data arrays of a geek_data live */
enum { GEEK_MEM_DEVICE = 0, GEEK_MEM_HOST = 1 };
/* dense projection family */
enum { GEEK_PROJ_E2LSH = 0, GEEK_PROJ_SRP = 1, GEEK_PROJ_QALSH = 2 };
/* arithmetic of the fast path (FP64 rechecks keep every result exact):
 * FP32 SIMT; BF16 tcgen05 (one product per term, error window ~2^-7 |x||c|);
 * split-BF16 tcgen05 (x = x_h + x_l, c = c_h + c_l in BF16 pairs, three
 * products x_h.c_h + x_l.c_h + x_h.c_l, window ~2^-14 |x||c|: far fewer
 * near-tie rechecks for three times the tensor work) */
enum { GEEK_PREC_FP32 = 0, GEEK_PREC_BF16 = 1, GEEK_PREC_BF16X3 = 2 };

/* One data set.
 *  DENSE : x is n x d float32, row-major with row stride ldx (elements).
 *  SETS  : set_off (n+1 int64, ascending, set_off[0] = 0) and set_items
 *          (uint32 item ids, distinct within a set) in CSR form.
 *  HETERO: x as DENSE for the numeric attributes plus cat, n x n_cat uint32
 *          tokens, row-major; token = offset of the attribute + value, so
 *          that different attributes never share a token (Alg. 2).
 * mem = GEEK_MEM_HOST marks x / set_off / set_items / cat as host memory
 * (pinned for speed): the library stages them to the device itself. */
typedef struct geek_data {
    int32_t kind;
    int32_t mem;
    int64_t n;
    int32_t d;
    int32_t n_cat;
    int64_t ldx;
    const float *x;
    const int64_t *set_off;
    const uint32_t *set_items;
    const uint32_t *cat;
} geek_data;

/* Hash parameters (Sect. 2.2 static (K,L) framework; Sect. 3.1, Algs. 2-3).
 *  Dense / hetero numeric part: F = K*L projections a (F x d float32,
 *    function f = l*K + k) and offsets b (F float32); E2LSH code =
 *    floor((a.x + b) / w) (the function named in Sect. 3.1 Remarks), or for
 *    proj = SRP the sign bit [a.x >= 0] (b and w unused).
 *  Sets: K*L MinHash functions (Eq. 2), coefficient pairs mh_a/mh_b (uint64),
 *    h(v) = ((mh_a*v + mh_b) mod 2^64) >> 32.
 *  Hetero: additionally Kc MinHash functions per table (Kc*L coefficient
 *    pairs) over each row's token set, appended to the table key.
 * Table l's key is the tuple of its K (+ Kc) values, compared
 * lexicographically (codes signed, MinHash values unsigned).
 *  proj = QALSH (Alg. 1, the paper's own transform of dense data): K = 1 and
 *    L = m tables, one per projection a_l (b and w unused); table l sorts
 *    the objects by s = a_l.x (the pinned FP64 dot product defined for
 *    E2LSH) with ties by ascending object id and cuts the sorted list into
 *    t buckets: bucket j holds sorted positions [floor(j n / t),
 *    floor((j + 1) n / t)), 1 <= t <= n.  codes then hold the FP32 bit
 *    patterns of the projections (approximate; the buckets are exact).
 *    DENSE data only; finite inputs.
 *  Sets with doph_bins = D' > 0 (Alg. 3's DOPH step, 1 <= D' <= 1024):
 *    pi(v) = ((doph_a*v + doph_b) mod 2^64) >> 32 cut into D' equal bins,
 *    bin(v) = (pi(v)*D') >> 32, offset(v) = (pi(v)*D') mod 2^32; a bin keeps
 *    its smallest offset; an empty bin takes the value of the first
 *    non-empty bin to its right (circular) at distance t (rotation
 *    densification); an empty set: t = D', value 2^32 - 1.  The set is
 *    replaced by its D' tokens (b << 48) | (t << 32) | value and the K*L
 *    MinHash functions hash the 64-bit tokens: ((mh_a*x + mh_b) mod 2^64)
 *    >> 32. */
typedef struct geek_hash_params {
    int32_t proj;
    int32_t precision;
    int32_t K, L, Kc;
    double w;
    const float *a;
    const float *b;
    const uint64_t *mh_a;
    const uint64_t *mh_b;
    int32_t t;           /* QALSH: buckets per table (ignored otherwise) */
    int32_t doph_bins;   /* SETS: > 0 reduces every set by DOPH to this many tokens first */
    uint64_t doph_a, doph_b;  /* SETS with doph_bins: the permutation hash pair */
} geek_hash_params;

typedef struct geek_buckets_info {
    int64_t n;               /* objects */
    int32_t L;               /* tables */
    int32_t key_bits_max;    /* widest packed table key, bits */
    int64_t n_buckets;       /* buckets over all tables */
    int64_t n_flagged;       /* elements outside the FP32 window (rechecked) */
    int64_t n_flagged_fp64;  /* of those, elements decided by the FP64 reference */
} geek_buckets_info;

/* SILK parameters (Alg. 4): Ls tables of Ks MinHash functions over object
 * ids (mh_a/mh_b, Ls*Ks pairs, function t*Ks + k), seeding threshold delta
 * (>= 1) and Ks functions dd_a/dd_b for the near-duplicate removal pass.
 * Device arrays.  1 <= Ks <= 4. */
typedef struct silk_params {
    int32_t Ks, Ls, delta;
    const uint64_t *mh_a, *mh_b;
    const uint64_t *dd_a, *dd_b;
} silk_params;

typedef struct geek_assign_params {
    int32_t precision; /* GEEK_PREC_FP32 (SIMT), GEEK_PREC_BF16 or GEEK_PREC_BF16X3 (tcgen05) */
} geek_assign_params;

typedef struct geek_assign_stats {
    double sse;              /* sum over objects of the distance to its centre */
    double radius_max;       /* max over objects of that distance (Sect. 4.1) */
    int64_t k;               /* number of centres used */
    int64_t n_recheck_rows;  /* objects the fast pass left undecided (then decided exactly) */
    int64_t n_fp64_rows;     /* of those, objects decided by the FP64 reference distance */
} geek_assign_stats;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (made current).  One context per
 * thread at a time; contexts are independent. */
geek_status geek_ctx_create(int device, geek_ctx **out);
geek_status geek_ctx_destroy(geek_ctx *ctx);
/* Context options (geek_ctx_set_option).  The paper has no counterpart:
 * these bound the library's own device waits and inject failures so that the
 * error paths can be tested without faulting a GPU.
 *  GEEK_OPT_WAIT_LIMIT_NS: limit of one bounded wait of a radix-sort pass on a
 *    predecessor tile's published count, in ns (default 2e9, range
 *    [1e3, 6e10]).  A wait that runs out gives up with a partial prefix (the
 *    pass's writes stay inside its segment; its result is wrong), and the
 *    call that sorted returns GEEK_ERR_TIMEOUT.
 *  GEEK_OPT_TEST_STALL_TILE: FOR TESTS.  Tile t >= 0 of every radix pass never
 *    publishes its count, so the tiles after it wait until the wait limit and
 *    the call returns GEEK_ERR_TIMEOUT; -1 (default) turns it off.
 *  GEEK_OPT_TEST_FAIL_ALLOC: FOR TESTS.  Value v >= 0 makes the device
 *    allocation after the next v ones fail as if the device were out of memory
 *    (the call returns GEEK_ERR_NOMEM, the countdown then turns itself off);
 *    -1 (default) turns it off.
 * Errors: INVALID (NULL ctx, unknown option, value out of range). */
enum { GEEK_OPT_WAIT_LIMIT_NS = 1, GEEK_OPT_TEST_STALL_TILE = 2, GEEK_OPT_TEST_FAIL_ALLOC = 3 };
geek_status geek_ctx_set_option(geek_ctx *ctx, int32_t option, int64_t value);
/* Message for the last failing call on ctx (never NULL; owned by ctx). */
const char *geek_last_error(const geek_ctx *ctx);
/* Library version string (static storage). */
const char *geek_version(void);

/* ---- resident data ------------------------------------------------------ */

/* A device copy of a host data set, owned by the library, that several calls
 * share (hash, SILK and assignment all read x: staging a host data set once
 * instead of once per call).
 * geek_data_upload copies `host` (mem = GEEK_MEM_HOST: x n*ldx floats,
 * set_off n+1 and set_items set_off[n] entries, cat n*n_cat tokens) into the
 * device buffers of *res, creating the handle when *res is NULL and growing
 * its buffers when they are too small, all in stream order on `stream`;
 * *view then describes the copy (mem = GEEK_MEM_DEVICE, same kind, n, d,
 * ldx and n_cat) and stays valid until the next upload into, or the free of,
 * the same handle.  The host arrays must stay unchanged until the copies
 * have completed (synchronise `stream`).
 * Errors: INVALID (NULL arguments, data not on the host, bad shapes), NOMEM,
 * CUDA.  On error *res keeps its previous buffers. */
typedef struct geek_resident geek_resident;
geek_status geek_data_upload(geek_ctx *ctx, const geek_data *host, geek_resident **res, geek_data *view,
                             geek_stream stream);
geek_status geek_resident_free(geek_resident *r);

/* ---- data transformation (Sect. 3.1) ------------------------------------ */

/* geek_hash: converts every object into one bucket per table.
 * Dense: E2LSH codes floor((a.x+b)/w) (or SRP bits) of K functions per table
 * over L tables.  Sets: MinHash (Eq. 2) K per table.  Hetero: E2LSH of the
 * numeric part followed by Kc MinHash values of the tokens (Alg. 2).
 * Exact definition of a code: s = sum_j (double)a_j*(double)x_j accumulated
 * in j order in FP64, code = floor((s + (double)b) / w) with IEEE
 * round-to-nearest; elements whose FP32 value lies within its rigorous
 * error bound of a code boundary are recomputed that way on the GPU.
 * Buckets of a table are the classes of equal keys; the canonical bucket id
 * of an object in table l is the rank of its key among table l's distinct
 * keys in ascending lexicographic order.  On success *out owns the result.
 * Errors: INVALID (shapes, K*L > 4096, Kc without HETERO), OVERFLOW (a code
 * outside int32 or a table key wider than 128 bits), NOMEM, CUDA. */
geek_status geek_hash(geek_ctx *ctx, const geek_data *data, const geek_hash_params *p,
                      geek_buckets **out, geek_stream stream);

geek_status geek_buckets_info_get(const geek_buckets *b, geek_buckets_info *info);

/* Copies results into caller device buffers (each pointer may be NULL):
 *  obj_bucket  L x n int32: canonical bucket id of object i in table l
 *  n_buckets   L int64 (HOST): buckets per table
 *  bucket_off  n_buckets_total + 1 int64: bucket g (tables concatenated in
 *              order, ranks ascending) holds members[bucket_off[g] ..
 *              bucket_off[g+1])
 *  members     L*n int32: object ids grouped by bucket, ascending inside
 *  codes       n x (K*L) int32: per-function codes (dense / hetero; for SETS
 *              the MinHash values as uint32 bit patterns) */
geek_status geek_buckets_copy_out(const geek_buckets *b, int32_t *obj_bucket, int64_t *n_buckets,
                                  int64_t *bucket_off, int32_t *members, int32_t *codes,
                                  geek_stream stream);
/* Releases b.  Its device memory was allocated, and is freed, in stream
 * order on the stream geek_hash ran on (no device-wide synchronisation):
 * that stream must still exist, and work reading b on other streams must
 * be complete. */
geek_status geek_buckets_free(geek_buckets *b);

/* ---- initial seeding, SILK (Sect. 3.2, Alg. 4) -------------------------- */

/* silk_seed: groups similar buckets into bins with Ls tables of Ks MinHash
 * functions over object ids; bins holding at most one bucket are skipped;
 * each other bin yields C_shared = the objects present in more than half of
 * its buckets (2*count > |bin|), kept when |C_shared| >= delta.  The
 * multiset of kept sets is then deduplicated with one more table of Ks
 * functions: a bin holding one set keeps it; a bin of several sets yields
 * their majority-vote set if it has >= delta objects, else its member that
 * is smallest in canonical order.  Exact duplicates are dropped and the
 * seeds sorted in canonical order (lexicographic on ascending member
 * lists); seed j is the j-th in that order.  k is an output, never input. */
geek_status silk_seed(geek_ctx *ctx, const geek_buckets *b, const silk_params *p,
                      silk_seeds **out, geek_stream stream);
/* k = number of seeds, n_ids = total members, n_multiset = kept C_shared
 * sets before near-duplicate removal (all HOST outputs). */
geek_status silk_seeds_info(const silk_seeds *s, int64_t *k, int64_t *n_ids, int64_t *n_multiset);
/* off: k+1 int64, ids: n_ids int32 (device buffers). */
geek_status silk_seeds_copy_out(const silk_seeds *s, int64_t *off, int32_t *ids, geek_stream stream);
/* Releases s, in stream order on the stream silk_seed ran on (the same
 * conditions as geek_buckets_free). */
geek_status silk_seeds_free(silk_seeds *s);

/* ---- data assignment (Sect. 3.3, Eq. 1) --------------------------------- */

/* geek_assign: builds the central vector of every seed and assigns every
 * object to its closest one, once.
 *  DENSE: centroid = (sum over members in ascending id of (double)x) /
 *    count; distance = sum_j ((double)x_j - c_j)^2 accumulated in j order in
 *    FP64 without fused multiply-add; label = argmin, ties to the smallest
 *    seed index.  The fast path (FP32 SIMT or BF16 tcgen05) keeps the best
 *    and second-best approximate distance per object; objects whose gap is
 *    within the rigorous error window are decided in FP64.
 *  HETERO: unified categorical attributes (per table, the bucket of the
 *    numeric E2LSH part; then the tokens); central vector = per-attribute
 *    mode (most frequent value, ties to the smallest); distance 1 - Jaccard,
 *    i.e. the label maximises the number of matching attributes.
 *  SETS: central vector = items present in more than half of the members;
 *    label maximises |A n C| / |A u C| (exact rational comparison).
 * labels: n int32.  centers (nullable, DENSE only): k x d float64 out.
 * stats (nullable, HOST): filled after the stream has finished the call. */
geek_status geek_assign(geek_ctx *ctx, const geek_data *data, const geek_buckets *b,
                        const silk_seeds *s, const geek_assign_params *p, int32_t *labels,
                        double *centers, geek_assign_stats *stats, geek_stream stream);

/* geek_cluster_radius: the radius of every cluster (Sect. 4.1 reports the
 * radius of the clusters): radius[j] = sqrt(max over objects i with
 * labels[i] == j of sum_t (x_it - c_jt)^2), 0 for a cluster with no object.
 * DENSE device data only; centers k x d float64, labels n int32 (values
 * outside [0, k) are skipped) and radius k float64 are device buffers.  The
 * distances are those of geek_assign_stats (FP32 with the centres split into
 * two FP32 parts, within 1e-6 relative of the FP64 value).  Stream-ordered,
 * no host synchronisation.  Errors: INVALID (NULL arguments, data not DENSE
 * or in host memory, k out of range), NOMEM, CUDA. */
geek_status geek_cluster_radius(geek_ctx *ctx, const geek_data *data, const double *centers, int64_t k,
                                const int32_t *labels, double *radius, geek_stream stream);

/* geek_assign_ex: geek_assign, and the central vectors it used (Sect. 3.3) kept
 * in a library-owned handle *centres (sizes vary with the data):
 *  DENSE: centers k x d float64 (the FP64 centroids).
 *  HETERO: modes k x n_attr int64, n_attr = L + n_cat: attribute l < L is
 *    the canonical rank of the mode's numeric E2LSH tuple among table l's
 *    distinct numeric tuples (ascending lexicographic order, as bucket ids);
 *    attribute L + j is the mode token of categorical attribute j (the value
 *    given in geek_data.cat).  Mode = most frequent value, ties to the
 *    smallest (in tuple order for the numeric attributes).
 *  SETS: centre j = items item_off[j] .. item_off[j+1] (ascending u32) of
 *    items, the items present in more than half of seed j's member sets.
 * Same arguments and errors as geek_assign otherwise (centers output dropped:
 * the handle holds it).  geek_centres_info_get gives kind, k, d (DENSE),
 * n_attr (HETERO) and n_items (SETS); geek_centres_copy_out copies the
 * arrays of the handle's kind into caller device buffers (NULL skips one);
 * geek_centres_free releases the handle. */
typedef struct geek_centres geek_centres;
typedef struct geek_centres_info {
    int32_t kind;
    int32_t d;
    int32_t n_attr;
    int64_t k;
    int64_t n_items;
} geek_centres_info;
geek_status geek_assign_ex(geek_ctx *ctx, const geek_data *data, const geek_buckets *b, const silk_seeds *s,
                           const geek_assign_params *p, int32_t *labels, geek_assign_stats *stats,
                           geek_centres **centres, geek_stream stream);
geek_status geek_centres_info_get(const geek_centres *c, geek_centres_info *info);
geek_status geek_centres_copy_out(const geek_centres *c, double *centers, int64_t *modes, int64_t *item_off,
                                  uint32_t *items, geek_stream stream);
geek_status geek_centres_free(geek_centres *c);

/* geek_refine: further passes of assignment for more compact clusters
 * (Sect. 5: several passes of data assignment; each pass is Lloyd's update
 * step then the assignment step, Sect. 2).  Dense data only.  On entry
 * labels (n int32, device) hold an assignment of the objects to the k
 * centres in centers (k x d float64, device), e.g. geek_assign's output.
 * Each pass replaces centre j by the FP64 mean of the objects labelled j
 * (summed in ascending object id, as the seeds' centroids; a centre with no
 * object keeps its value) and then reassigns every object with the exact
 * argmin of geek_assign_centers (precision p->precision).  centers and
 * labels are updated in place; stats (nullable, HOST) describe the last
 * assignment.  passes >= 0; labels must lie in [-1, k).
 * Errors: INVALID (NULL arguments, data not DENSE, passes < 0, a label
 * outside [-1, k)), NOMEM, CUDA. */
geek_status geek_refine(geek_ctx *ctx, const geek_data *data, double *centers, int64_t k, int32_t passes,
                        const geek_assign_params *p, int32_t *labels, geek_assign_stats *stats,
                        geek_stream stream);

/* geek_assign_centers: the dense assignment of geek_assign against k given
 * central vectors (k x d float64, device), with the same exact argmin
 * definition.  Useful when the centres come from elsewhere. */
geek_status geek_assign_centers(geek_ctx *ctx, const geek_data *data, const double *centers,
                                int64_t k, const geek_assign_params *p, int32_t *labels,
                                geek_assign_stats *stats, geek_stream stream);

/* ---- allocation-free dense assignment ------------------------------------ */

/* The paper has no counterpart of this entry point: it serves callers that
 * cannot allocate device memory during the call, for example a serving loop
 * whose memory is fully reserved up front by another allocator (a framework's
 * caching pool holding all free memory, where cudaMalloc would fail), or code
 * that must not pay the device-wide synchronisation an allocation or free
 * can imply.
 *
 * geek_assign_centers_noalloc computes exactly what geek_assign_centers
 * computes with GEEK_PREC_FP32 (same labels: the FP64 nearest centre, ties
 * to the smallest index) but allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch (the FP32 centres and their norms)
 * is one fixed device array of GEEK_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads this library holds until the process exits.  Arguments are device
 * pointers on the current device: x (n x d float32, row stride ldx), centers
 * (k x d float64), labels (n int32, also used to mark undecided rows while the
 * call runs).  No context is needed; the call is stream-ordered on `stream`.
 *  - The first call on a device does a one-time set-up with that device
 *    current (it looks up the scratch array's device address); make that
 *    first call before any stream capture.
 *  - Every call shares the one scratch array and leaves the last call's
 *    contents in it: calls that overlap on the GPU (different streams or
 *    threads without ordering) race and give wrong results.
 *  - Returns GEEK_ERR_INVALID for bad arguments and GEEK_ERR_UNSUPPORTED when
 *    d > 256, k > GEEK_NOALLOC_MAX_K or k*d > GEEK_NOALLOC_MAX_KD (the
 *    scratch limit); GEEK_ERR_CUDA if a CUDA call or launch fails, and also,
 *    without launching anything, when an earlier CUDA error is still
 *    pending on the calling thread (it is left pending for its owner). */
#define GEEK_NOALLOC_MAX_K 65536
#define GEEK_NOALLOC_MAX_KD 1048576
#define GEEK_NOALLOC_SCRATCH_BYTES (4 * GEEK_NOALLOC_MAX_KD + 4 * GEEK_NOALLOC_MAX_K + 256)
geek_status geek_assign_centers_noalloc(const float *x, int64_t n, int32_t d, int64_t ldx,
                                        const double *centers, int64_t k, int32_t *labels,
                                        geek_stream stream);

/* ---- batched instances ------------------------------------------------------ */

/* Many independent dense clustering problems of uneven n, d and seed count run
 * as one batch: the whole pipeline above (E2LSH / SRP hashing, bucket grouping,
 * SILK seeding, centroids and the one-pass assignment, Sects. 3.1-3.3) for every
 * instance, with each step launched once for all instances.  The hashing pass
 * runs every instance's row blocks in one launch and the BF16 tcgen05 assignment
 * runs all (instance, row tile) units in one persistent launch; both phases are
 * captured in CUDA graphs on the first run and replayed by later runs.  The
 * assignment's arithmetic (BF16 or split-BF16) and centre-tile width (64, 128
 * or 256 columns) are chosen per instance by an autotuner that times the
 * candidates, FP64 near-tie decisions included, on the batch's own data the
 * first time a (d, seed count) class is seen on a context.
 * Results are, instance by instance, exactly those of geek_hash + silk_seed +
 * geek_assign on that instance alone (every precision gives the same,
 * exact labels). */
typedef struct geek_batch geek_batch;

/* One dense instance: x (n x d float32, row stride ldx, n >= 0, 1 <= d <= 128),
 * its K*L projections a (K*L x d float32) and offsets b (K*L float32), bucket
 * width w (E2LSH), and its SILK coefficients mh_a/mh_b (Ls*Ks pairs) and
 * dd_a/dd_b (Ks pairs) as in silk_params.  Device arrays; they must stay
 * valid, at the same addresses, for the life of the batch (their contents
 * may change between runs). */
typedef struct geek_instance {
    int64_t n;
    int32_t d;
    int64_t ldx;
    const float *x;
    const float *a;
    const float *b;
    double w;
    const uint64_t *mh_a, *mh_b;
    const uint64_t *dd_a, *dd_b;
} geek_instance;

/* Shared by every instance: projection family, K functions per table, L
 * tables, SILK Ks / Ls / delta; the assignment's arithmetic, precision =
 * GEEK_PREC_BF16, GEEK_PREC_BF16X3 or GEEK_PREC_AUTO (the autotuner picks one
 * per class of instances: the fewer tensor products of BF16 against the
 * fewer FP64 near-tie decisions of split-BF16); tile_n: 0 = autotuned, or
 * 64 / 128 / 256 to force the centre-tile width (split-BF16 caps it at 128
 * for d <= 64 and 64 for d <= 128). */
#define GEEK_PREC_AUTO (-1)
typedef struct geek_batch_params {
    int32_t proj;
    int32_t K, L;
    int32_t Ks, Ls, delta;
    int32_t precision;
    int32_t tile_n;
} geek_batch_params;

typedef struct geek_batch_info {
    int32_t count;            /* instances */
    int64_t n_total;          /* objects over all instances */
    int64_t k_total;          /* seeds over all instances (last run) */
    int64_t n_buckets;        /* buckets over all instances and tables */
    int64_t n_flagged;        /* projection elements rechecked */
    int64_t n_flagged_fp64;   /* of those, decided by the FP64 reference */
    int64_t n_recheck_rows;   /* objects the fast assignment pass left undecided */
    int32_t key_bits;         /* composite sort key width (instance id + key) */
    int32_t graph_launches;   /* CUDA graph replays so far (hash + assignment) */
    int32_t graph_captures;   /* graphs captured so far */
    int32_t tuned_classes;    /* (d, k) classes this batch timed for tile_n */
    int64_t n_fp64_rows;      /* of the undecided objects, those decided by the FP64 reference */
} geek_batch_info;

/* Creates a batch of `count` (1..65535) instances; validates the parameters
 * and sets up the hashing phase (nothing runs yet).  Instances are numbered
 * 0..count-1 and their objects concatenated in that order (global row
 * r = sum of earlier n + local row).  Errors: INVALID, UNSUPPORTED (d > 128,
 * more than 2^31 - 1 objects, K*L > 512), NOMEM, CUDA. */
geek_status geek_batch_create(geek_ctx *ctx, const geek_instance *inst, int32_t count,
                              const geek_batch_params *p, geek_batch **out);

/* Runs the whole pipeline for every instance on `stream`.  labels: n_total
 * int32 (device), instance i's labels at its global rows, as seed indices
 * local to the instance (0..k_i-1, or -1 when the instance has no seed).
 * Returns after the run has finished on the device (the seed counts it
 * needs are read back mid-way).  Calls on one batch must not overlap. */
geek_status geek_batch_run(geek_batch *b, int32_t *labels, geek_stream stream);

geek_status geek_batch_info_get(const geek_batch *b, geek_batch_info *info);

/* Per-instance results of the last run, HOST arrays of `count` entries (each
 * pointer may be NULL): seed count k, SSE and largest distance to the
 * assigned centre (Sect. 4.1), and the assignment's centre-tile width and
 * precision (GEEK_PREC_BF16 or GEEK_PREC_BF16X3). */
geek_status geek_batch_instance_stats(const geek_batch *b, int64_t *k, double *sse, double *radius_max,
                                      int32_t *tile_n, int32_t *precision);

/* Device copies of the last run's intermediate results (each pointer may be
 * NULL):
 *  codes       n_total x (K*L) int32 per-function codes
 *  obj_bucket  L x n_total int32: per instance, the canonical bucket id of
 *              geek_hash on that instance alone (ranks restart at 0)
 *  seed_off    k_total + 1 int64 and seed_ids (int32, local ids): the seeds
 *              of all instances in instance order, each instance's in its
 *              canonical order
 *  centres     sum_i k_i * d_i float64: instance i's k_i x d_i centroids,
 *              instances in order */
geek_status geek_batch_copy_out(const geek_batch *b, int32_t *codes, int32_t *obj_bucket, int64_t *seed_off,
                                int32_t *seed_ids, double *centres, geek_stream stream);
/* Seed id count of the last run (the size of seed_ids). */
geek_status geek_batch_seed_ids_count(const geek_batch *b, int64_t *n_ids);
geek_status geek_batch_destroy(geek_batch *b);

/* ---- tracing -------------------------------------------------------------- */

/* When on, every phase (names "hash", "silk", "assign") and the main kernels
 * are bracketed by CUDA events on the call's stream; each bracket waits for
 * its end event, so timing adds synchronisation.  Off by default.  Kernel
 * brackets also record their algorithmic work: "kernel.project_fp32" and
 * "kernel.assign_fp32" / "kernel.assign_tc" in flops (2 d per output element),
 * "kernel.recheck_fp64" in FP64 flops (2 d per rechecked element),
 * "kernel.rs_scatter" in bytes (each key word, and the value, read once and
 * written once); "hash.sort" and "kernel.assign_recheck" record time only. */
geek_status geek_timing_enable(geek_ctx *ctx, int on);
geek_status geek_timing_reset(geek_ctx *ctx);
/* Total milliseconds, bracket count and recorded work under `name` (0 if
 * none).  Any output pointer may be NULL. */
geek_status geek_timing_get(const geek_ctx *ctx, const char *name, double *total_ms, int64_t *count,
                            double *total_work);
/* Kernels launched by this library in this process so far. */
unsigned long long geek_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GEEK_H */
