"""FP64 / exact CPU oracle for GEEK hashing, SILK seeding and assignment.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to check and time the GPU library; the library itself
never imports it.  The arithmetic lives in ``geek_oracle.c`` (plain C, built
with ``-O2 -ffp-contract=off`` and OpenMP over independent objects); this
module marshals NumPy arrays and composes the steps in the paper's order:

* dense data (Sect. 3.1): E2LSH codes floor((a.x+b)/w) (or sign bits), K per
  table concatenated over L tables (the static (K,L) framework, Sect. 2.2);
* dense data, the paper's own transform (Alg. 1): m QALSH projections a.x,
  each table sorted (ties by object id) and split evenly into t buckets;
* sparse sets (Alg. 3): MinHash (Eq. 2), K per table, L tables, on the sets
  themselves or (transform_sparse_doph) on their DOPH reduction;
* heterogeneous rows (Alg. 2): E2LSH codes of the numeric part concatenated
  with MinHash of the categorical tokens, per table;
* SILK (Alg. 4) with majority voting and near-duplicate removal;
* central vectors (Sect. 3.3) and one-pass assignment (Eq. 1);
* further passes of assignment (Sect. 5: several passes for more compact
  clusters), each an update of the centres then a reassignment.

Parity status of each function is listed in ``PINS`` below.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geek_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgeek_oracle.so")
_lib = None

# What pins each oracle function to something other than itself (the tests
# under tests/test_oracle_*.py implement every item).
PINS = {
    "e2lsh": "exact rational floor((a.x+b)/w) with fractions.Fraction (brute force)",
    "srp": "exact rational sign of a.x (brute force)",
    "alg1": "exact rational projections sorted by (value, id) and split by floor(b n / t) (brute force); "
            "bucket sizes, tie order and the t = 1 / t = n cases",
    "hash32": "Python big-integer (A*x+B) mod 2^64 >> 32",
    "doph": "hand-worked bins, borrowing and wrap-around with an affine pi; per-bin collision rate = Jaccard "
            "(rotation densification); 64-bit-token MinHash against Python big integers",
    "minhash": "explicit set minima in Python; collision rate = Jaccard (Eq. 2)",
    "group": "Python dict of tuples, canonical rank by sorted distinct keys",
    "vote": "Example 2 with forced bins (Sect. 3.2)",
    "silk": "Python brute-force re-statement on tiny inputs + invariants",
    "centroids": "exact rational mean within 1 ulp",
    "assign_dense": "exhaustive exact-rational nearest seed",
    "refine_passes": "separated blobs: exact rational blob means after one pass; SSE non-increasing; "
                     "fixed point; a centre without members keeps its value",
    "hash_hetero": "per-table key rebuilt from exact rational codes and big-integer MinHash, grouped with dicts",
    "hetero_attrs": "per-table rank of the numeric tuple among sorted distinct tuples, then the raw values",
    "modes": "collections.Counter brute force",
    "assign_cat": "brute-force match counts",
    "sparse_centres": "Counter brute force",
    "doph_modes": "Counter brute force per reduced dimension over hand-built DOPH tokens",
    "assign_doph": "brute-force count of dimensions equal to each mode",
    "assign_jaccard": "fractions.Fraction brute force",
}


def build(force: bool = False) -> str:
    """Compile geek_oracle.c into a shared library (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                           "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.c_void_p
        i64, i32, f64 = C.c_int64, C.c_int32, C.c_double
        L.orc_e2lsh.argtypes = [i64, i32, P, i64, i32, P, P, f64, P]
        L.orc_srp.argtypes = [i64, i32, P, i64, i32, P, P]
        L.orc_qalsh.argtypes = [i64, i32, P, i64, i32, P, P]
        L.orc_hash32.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32]
        L.orc_hash32.restype = C.c_uint32
        L.orc_minhash_csr.argtypes = [i64, P, P, i32, P, P, P]
        L.orc_doph.argtypes = [i64, P, P, i32, C.c_uint64, C.c_uint64, P]
        L.orc_minhash_rows64.argtypes = [i64, i32, P, i32, P, P, P]
        L.orc_sort_rows.argtypes = [i64, i32, P, P]
        L.orc_group.argtypes = [i64, i32, i32, P, P, P, P, P]
        L.orc_bucket_sigs.argtypes = [i64, P, P, i32, P, P, P]
        L.orc_vote_bins.argtypes = [i64, P, P, P, P, i32, P, P]
        L.orc_silk.argtypes = [i64, P, P, i32, i32, i32, P, P, P, P, P, P, P, P]
        L.orc_dedup_bins.argtypes = [i64, P, P, i64, P, P, i32, P, P, P]
        L.orc_free.argtypes = [P]
        L.orc_centroids.argtypes = [i64, i32, P, i64, i64, P, P, P]
        L.orc_assign_dense.argtypes = [i64, i32, P, i64, i64, P, P, P]
        L.orc_modes.argtypes = [i64, i32, P, i64, P, P, P]
        L.orc_assign_cat.argtypes = [i64, i32, P, i64, P, P, P]
        L.orc_sparse_centres.argtypes = [P, P, i64, P, P, P, P]
        L.orc_assign_jaccard.argtypes = [i64, P, P, i64, P, P, P, P, P]
        L.orc_num_threads.restype = C.c_int
    return _lib


def threads() -> int:
    return int(lib().orc_num_threads())


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else C.c_void_p(0)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# ---------------------------------------------------------------- hashing --
def e2lsh(x, a, b, w):
    """codes[i, f] = floor((a_f . x_i + b_f) / w) (pinned FP64 sequence)."""
    x = _c(x, np.float32); a = _c(a, np.float32); b = _c(b, np.float32)
    n, d = x.shape
    F = a.shape[0]
    out = np.empty((n, F), dtype=np.int32)
    _chk(lib().orc_e2lsh(n, d, _p(x), d, F, _p(a), _p(b), float(w), _p(out)), "e2lsh")
    return out


def srp(x, a):
    """bits[i, f] = [a_f . x_i >= 0]."""
    x = _c(x, np.float32); a = _c(a, np.float32)
    n, d = x.shape
    F = a.shape[0]
    out = np.empty((n, F), dtype=np.uint8)
    _chk(lib().orc_srp(n, d, _p(x), d, F, _p(a), _p(out)), "srp")
    return out


def hash32(A, B, x) -> int:
    return int(lib().orc_hash32(int(A), int(B), int(x)))


def minhash_csr(off, items, A, B):
    """out[i, f] = min over the items of set i of h_f(item)."""
    off = _c(off, np.int64); items = _c(items, np.uint32)
    A = _c(A, np.uint64); B = _c(B, np.uint64)
    n = off.size - 1
    out = np.empty((n, A.size), dtype=np.uint32)
    _chk(lib().orc_minhash_csr(n, _p(off), _p(items), A.size, _p(A), _p(B), _p(out)), "minhash")
    return out


def minhash_rows(tokens, A, B):
    """MinHash of fixed-length token rows (each row a set of tokens)."""
    tokens = _c(tokens, np.uint32)
    n, m = tokens.shape
    off = np.arange(n + 1, dtype=np.int64) * m
    return minhash_csr(off, tokens.reshape(-1), A, B)


def doph(off, items, Dp, Ap, Bp):
    """DOPH reduction (Alg. 3's first step): n x Dp 64-bit tokens."""
    off = _c(off, np.int64); items = _c(items, np.uint32)
    n = off.size - 1
    out = np.empty((n, Dp), dtype=np.uint64)
    _chk(lib().orc_doph(n, _p(off), _p(items), int(Dp), int(Ap), int(Bp), _p(out)), "doph")
    return out


def minhash_rows64(tokens, A, B):
    tokens = _c(tokens, np.uint64); A = _c(A, np.uint64); B = _c(B, np.uint64)
    n, m = tokens.shape
    out = np.empty((n, A.size), dtype=np.uint32)
    _chk(lib().orc_minhash_rows64(n, m, _p(tokens), A.size, _p(A), _p(B), _p(out)), "minhash64")
    return out


def transform_sparse_doph(off, items, Dp, Ap, Bp, A, B, K, L):
    """Alg. 3 with its DOPH step: reduce every set to Dp tokens, then MinHash
    (K, L) on the reduced sets and group per table."""
    tok = doph(off, items, Dp, Ap, Bp)
    mh = minhash_rows64(tok, A, B)
    return tok, mh, group(table_keys(mh, L, K))


# --------------------------------------------------------------- grouping --
class Buckets:
    """Per-table canonical bucketing.  obj_bucket[l, i] = rank of object i's
    key among table l's distinct keys (ascending lexicographic order);
    tables' buckets are numbered consecutively for SILK (global id =
    table_base[l] + rank) with members ascending inside each bucket."""

    def __init__(self, obj_bucket, n_buckets, members, bucket_off):
        self.obj_bucket = obj_bucket
        self.n_buckets = n_buckets
        self.L, self.n = obj_bucket.shape
        self.table_base = np.concatenate([[0], np.cumsum(n_buckets)[:-1]]).astype(np.int64)
        self.NB = int(n_buckets.sum())
        offs = []
        for l in range(self.L):
            offs.append(bucket_off[l, : n_buckets[l]] + l * self.n)
        self.boff = np.concatenate(offs + [np.array([self.L * self.n])]).astype(np.int64)
        self.bmem = members.reshape(-1).astype(np.int32)

    def sizes(self):
        return np.diff(self.boff)


def group(keys):
    """keys: int64 [L, n, W] -> Buckets."""
    keys = _c(keys, np.int64)
    L, n, W = keys.shape
    ob = np.empty((L, n), dtype=np.int32)
    nb = np.empty(L, dtype=np.int64)
    mem = np.empty((L, n), dtype=np.int32)
    bo = np.empty((L, n + 1), dtype=np.int64)
    _chk(lib().orc_group(n, L, W, _p(keys), _p(ob), _p(nb), _p(mem), _p(bo)), "group")
    return Buckets(ob, nb, mem, bo)


def table_keys(codes, L, K):
    """[n, L*K] codes (function f = l*K + k) -> int64 keys [L, n, K]."""
    n = codes.shape[0]
    return np.ascontiguousarray(codes.reshape(n, L, K).transpose(1, 0, 2).astype(np.int64))


def hash_dense(x, a, b, w, K, L, proj="e2lsh"):
    codes = e2lsh(x, a, b, w) if proj == "e2lsh" else srp(x, a).astype(np.int32)
    return codes, group(table_keys(codes, L, K))


def qalsh(x, a):
    """s[i, f] = a_f . x_i (pinned FP64 sequence), the QALSH value of Alg. 1."""
    x = _c(x, np.float32); a = _c(a, np.float32)
    n, d = x.shape
    m = a.shape[0]
    out = np.empty((n, m), dtype=np.float64)
    _chk(lib().orc_qalsh(n, d, _p(x), d, m, _p(a), _p(out)), "qalsh")
    return out


def split_even(values, t):
    """One table of Alg. 1: objects sorted by (value, id) ascending, the
    sorted list cut into t parts; part b holds sorted positions
    [floor(b n / t), floor((b + 1) n / t)).  Returns the bucket of every
    object (ties between equal values go by ascending object id)."""
    n = values.shape[0]
    order = np.lexsort((np.arange(n), values))  # primary key: value, then id
    bucket_at = (np.arange(1, n + 1) * t + n - 1) // n - 1  # largest b with floor(b n / t) <= p
    ob = np.empty(n, dtype=np.int32)
    ob[order] = bucket_at
    return ob


def transform_alg1(x, a, t):
    """Alg. 1: m = rows of a QALSH functions, one table each, t buckets per
    table.  Returns (s, Buckets) with canonical bucket id = part index."""
    s = qalsh(x, a)
    n, m = s.shape
    if not 1 <= t <= max(n, 1):
        raise ValueError("need 1 <= t <= n")
    ob = np.empty((m, n), dtype=np.int32)
    nb = np.full(m, t, dtype=np.int64)
    mem = np.empty((m, n), dtype=np.int32)
    bo = np.zeros((m, n + 1), dtype=np.int64)
    cuts = (np.arange(t) * n) // t
    for f in range(m):
        ob[f] = split_even(s[:, f], t)
        mem[f] = np.argsort(ob[f], kind="stable")  # by bucket, ascending id inside
        bo[f, :t] = cuts
    return s, Buckets(ob, nb, mem, bo)


def hash_sets(off, items, A, B, K, L):
    mh = minhash_csr(off, items, A, B)
    return mh, group(table_keys(mh, L, K))


def hash_hetero(x, tokens, a, b, w, K, L, A, B, Kc):
    """Alg. 2 reading: per table, the K E2LSH codes of the numeric part
    followed by the Kc MinHash values of the categorical token set."""
    codes = e2lsh(x, a, b, w)
    mh = minhash_rows(tokens, A, B)
    n = x.shape[0]
    kc = table_keys(codes, L, K)
    km = table_keys(mh, L, Kc)
    keys = np.concatenate([kc, km], axis=2)
    return codes, mh, group(keys), group(kc)


def hetero_attrs(numeric_buckets, cat):
    """Unified categorical attributes of heterogeneous rows (Sect. 3.3): the
    canonical E2LSH-only bucket rank per table, then the raw categorical
    values.  int64 [n, L + n_cat]."""
    return np.concatenate([numeric_buckets.obj_bucket.T.astype(np.int64),
                           np.asarray(cat, dtype=np.int64)], axis=1)


# ------------------------------------------------------------------- SILK --
class Seeds:
    def __init__(self, off, ids, n_multiset):
        self.off, self.ids, self.n_multiset = off, ids, n_multiset
        self.k = off.size - 1

    def sets(self):
        return [tuple(self.ids[self.off[j]:self.off[j + 1]].tolist()) for j in range(self.k)]


def bucket_sigs(boff, bmem, A, B):
    boff = _c(boff, np.int64); bmem = _c(bmem, np.int32)
    A = _c(A, np.uint64); B = _c(B, np.uint64)
    NB = boff.size - 1
    out = np.empty((NB, A.size), dtype=np.uint32)
    _chk(lib().orc_bucket_sigs(NB, _p(boff), _p(bmem), A.size, _p(A), _p(B), _p(out)), "sigs")
    return out


def vote_bins(bins, buckets, delta):
    """Majority vote over explicit bins.  bins: list of lists of bucket
    indices into ``buckets`` (a list of member lists).  Returns C_shared per
    bin (empty tuple when skipped or below delta)."""
    boff = np.zeros(len(buckets) + 1, dtype=np.int64)
    boff[1:] = np.cumsum([len(b) for b in buckets])
    bmem = np.array([i for b in buckets for i in b], dtype=np.int32)
    bin_off = np.zeros(len(bins) + 1, dtype=np.int64)
    bin_off[1:] = np.cumsum([len(b) for b in bins])
    bin_bucket = np.array([g for b in bins for g in b], dtype=np.int64)
    out_off = np.zeros(len(bins) + 1, dtype=np.int64)
    out_ids = np.zeros(max(1, bmem.size), dtype=np.int32)
    _chk(lib().orc_vote_bins(len(bins), _p(bin_off), _p(bin_bucket), _p(boff), _p(bmem),
                             int(delta), _p(out_off), _p(out_ids)), "vote")
    return [tuple(out_ids[out_off[b]:out_off[b + 1]].tolist()) for b in range(len(bins))]


def _csr_out(k, so, si):
    off = np.ctypeslib.as_array(so, shape=(k + 1,)).copy()
    ids = np.ctypeslib.as_array(si, shape=(max(1, int(off[-1])),))[: int(off[-1])].copy()
    lib().orc_free(C.cast(so, C.c_void_p))
    lib().orc_free(C.cast(si, C.c_void_p))
    return off, ids


def dedup_bins(sets, bins, delta):
    """Near-duplicate removal on explicit bins of a seed multiset.  sets:
    list of ascending tuples; bins: list of lists of indices into sets.
    Returns the final seeds as a canonical list of tuples."""
    coff = np.zeros(len(sets) + 1, dtype=np.int64)
    coff[1:] = np.cumsum([len(s) for s in sets])
    cids = np.array([i for s in sets for i in s], dtype=np.int32)
    bin_off = np.zeros(len(bins) + 1, dtype=np.int64)
    bin_off[1:] = np.cumsum([len(b) for b in bins])
    bin_set = np.array([g for b in bins for g in b], dtype=np.int64)
    k = C.c_int64()
    so = C.POINTER(C.c_int64)(); si = C.POINTER(C.c_int32)()
    _chk(lib().orc_dedup_bins(len(sets), _p(coff), _p(cids), len(bins), _p(bin_off), _p(bin_set),
                              int(delta), C.byref(k), C.byref(so), C.byref(si)), "dedup")
    off, ids = _csr_out(k.value, so, si)
    return [tuple(ids[off[j]:off[j + 1]].tolist()) for j in range(k.value)]


def silk(boff, bmem, Ks, Ls, delta, mh_a, mh_b, dd_a, dd_b) -> Seeds:
    boff = _c(boff, np.int64); bmem = _c(bmem, np.int32)
    mh_a = _c(mh_a, np.uint64); mh_b = _c(mh_b, np.uint64)
    dd_a = _c(dd_a, np.uint64); dd_b = _c(dd_b, np.uint64)
    assert mh_a.size == Ks * Ls and dd_a.size == Ks
    k = C.c_int64(); nm = C.c_int64()
    so = C.POINTER(C.c_int64)(); si = C.POINTER(C.c_int32)()
    _chk(lib().orc_silk(boff.size - 1, _p(boff), _p(bmem), Ks, Ls, int(delta), _p(mh_a),
                        _p(mh_b), _p(dd_a), _p(dd_b), C.byref(k), C.byref(so), C.byref(si),
                        C.byref(nm)), "silk")
    off, ids = _csr_out(k.value, so, si)
    return Seeds(off, ids, nm.value)


def silk_on(buckets: Buckets, sp) -> Seeds:
    return silk(buckets.boff, buckets.bmem, sp["Ks"], sp["Ls"], sp["delta"],
                sp["mh_a"], sp["mh_b"], sp["dd_a"], sp["dd_b"])


# ------------------------------------------------------------- assignment --
def centroids(x, seeds: Seeds):
    x = _c(x, np.float32)
    n, d = x.shape
    c = np.empty((seeds.k, d), dtype=np.float64)
    _chk(lib().orc_centroids(n, d, _p(x), d, seeds.k, _p(seeds.off), _p(seeds.ids), _p(c)), "centroids")
    return c


def assign_dense(x, centres):
    x = _c(x, np.float32); centres = _c(centres, np.float64)
    n, d = x.shape
    k = centres.shape[0]
    lab = np.empty(n, dtype=np.int32)
    dist = np.empty(n, dtype=np.float64)
    _chk(lib().orc_assign_dense(n, d, _p(x), d, k, _p(centres), _p(lab), _p(dist)), "assign")
    return lab, dist


def update_centres(x, labels, centres):
    """One update of a pass: centre j = FP64 mean of the objects labelled j
    (summed in ascending object id, as for the seeds' centroids); a centre
    with no object keeps its value."""
    k = centres.shape[0]
    n = labels.shape[0]
    lab = np.asarray(labels, dtype=np.int64)
    keep = lab >= 0
    order = np.lexsort((np.arange(n), lab))  # by label, then id
    order = order[keep[order]]
    counts = np.bincount(lab[keep], minlength=k)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    means = centroids(x, Seeds(off, order.astype(np.int32), 0)) if k else np.zeros((0, x.shape[1]))
    out = np.array(centres, dtype=np.float64, copy=True)
    out[counts > 0] = means[counts > 0]
    return out


def refine_passes(x, centres, labels, passes):
    """Sect. 5's extra passes of assignment: update the centres from the
    current labels, then reassign every object (Eq. 1), `passes` times.
    Returns (labels, centres, dist) of the last pass."""
    c = np.array(centres, dtype=np.float64, copy=True)
    lab = np.asarray(labels, dtype=np.int32)
    dist = None
    for _ in range(passes):
        c = update_centres(x, lab, c)
        lab, dist = assign_dense(x, c)
    return lab, c, dist


def modes(attrs, seeds: Seeds):
    attrs = _c(attrs, np.int64)
    n, A = attrs.shape
    m = np.empty((seeds.k, A), dtype=np.int64)
    _chk(lib().orc_modes(n, A, _p(attrs), seeds.k, _p(seeds.off), _p(seeds.ids), _p(m)), "modes")
    return m


def assign_cat(attrs, modes_):
    attrs = _c(attrs, np.int64); modes_ = _c(modes_, np.int64)
    n, A = attrs.shape
    lab = np.empty(n, dtype=np.int32)
    mt = np.empty(n, dtype=np.int32)
    _chk(lib().orc_assign_cat(n, A, _p(attrs), modes_.shape[0], _p(modes_), _p(lab), _p(mt)), "assign_cat")
    return lab, mt


def sparse_centres(off, items, seeds: Seeds):
    off = _c(off, np.int64); items = _c(items, np.uint32)
    co = C.POINTER(C.c_int64)(); ci = C.POINTER(C.c_uint32)()
    _chk(lib().orc_sparse_centres(_p(off), _p(items), seeds.k, _p(seeds.off), _p(seeds.ids),
                                  C.byref(co), C.byref(ci)), "sparse_centres")
    coff = np.ctypeslib.as_array(co, shape=(seeds.k + 1,)).copy()
    tot = int(coff[-1])
    cit = np.ctypeslib.as_array(ci, shape=(max(1, tot),))[:tot].copy()
    lib().orc_free(C.cast(co, C.c_void_p))
    lib().orc_free(C.cast(ci, C.c_void_p))
    return coff, cit


def assign_jaccard(off, items, coff, citems):
    off = _c(off, np.int64); items = _c(items, np.uint32)
    coff = _c(coff, np.int64); citems = _c(citems, np.uint32)
    n = off.size - 1
    lab = np.empty(n, dtype=np.int32)
    inter = np.empty(n, dtype=np.int64)
    uni = np.empty(n, dtype=np.int64)
    _chk(lib().orc_assign_jaccard(n, _p(off), _p(items), coff.size - 1, _p(coff), _p(citems),
                                  _p(lab), _p(inter), _p(uni)), "assign_jaccard")
    return lab, inter, uni


def doph_modes(tokens, seeds: Seeds):
    """Central vector of sparse sets reduced by DOPH (Sect. 3.3: the mode of
    each reduced dimension): for every seed and dimension b, the most
    frequent token of its members (ties to the smallest).  int64 [k, D']."""
    return modes(np.asarray(tokens, dtype=np.uint64).view(np.int64), seeds)


def assign_doph(tokens, modes_):
    """One-pass assignment of DOPH-reduced sets (Eq. 1 with 1 - Jaccard of
    the token sets; every set and centre holds D' tokens, so the label
    maximises the number of dimensions equal to the mode, ties to the
    smallest seed index)."""
    return assign_cat(np.asarray(tokens, dtype=np.uint64).view(np.int64), modes_)


def subset_rows(off, items, rows):
    """CSR sub-collection of the given set indices (for sampled checks)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = off[rows + 1] - off[rows]
    noff = np.zeros(rows.size + 1, dtype=np.int64)
    noff[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows]) if rows.size else np.zeros(0, np.int64)
    return noff, items[idx]


# ---------------------------------------------------------- whole pipelines --
def run_workload(wl, assign_rows=None):
    """Hash -> SILK -> central vectors -> assignment for one synthetic
    workload (dict from ``synth.make``).  ``assign_rows`` restricts the
    assignment to a sample of objects (for full-size checks)."""
    cfg = wl["cfg"]
    res = {}
    if cfg.kind == "dense":
        codes, bk = hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
        res.update(codes=codes, buckets=bk)
    elif cfg.kind == "sets" and wl.get("doph"):
        dp = wl["doph"]
        tok, mh, bk = transform_sparse_doph(wl["set_off"], wl["set_items"], dp["bins"], dp["a"], dp["b"],
                                            wl["mh_a"], wl["mh_b"], cfg.K, cfg.L)
        res.update(codes=mh, buckets=bk, tokens=tok)
    elif cfg.kind == "sets":
        mh, bk = hash_sets(wl["set_off"], wl["set_items"], wl["mh_a"], wl["mh_b"], cfg.K, cfg.L)
        res.update(codes=mh, buckets=bk)
    else:
        codes, mh, bk, nbk = hash_hetero(wl["x"], wl["tokens"], wl["a"], wl["b"], wl["w"],
                                         cfg.K, cfg.L, wl["mh_a"], wl["mh_b"], cfg.Kc)
        res.update(codes=codes, mh=mh, buckets=bk, numeric_buckets=nbk)
    seeds = silk_on(res["buckets"], wl["silk"])
    res["seeds"] = seeds
    rows = np.arange(cfg.n) if assign_rows is None else np.asarray(assign_rows)
    res["rows"] = rows
    if seeds.k == 0:
        res["labels"] = np.full(rows.size, -1, dtype=np.int32)
        return res
    if cfg.kind == "dense":
        c = centroids(wl["x"], seeds)
        lab, dist = assign_dense(wl["x"][rows], c)
        res.update(centres=c, labels=lab, dist=dist)
    elif cfg.kind == "sets" and wl.get("doph"):
        m = doph_modes(res["tokens"], seeds)
        lab, mt = assign_doph(res["tokens"][rows], m)
        res.update(modes=m, labels=lab, matches=mt)
    elif cfg.kind == "sets":
        coff, cit = sparse_centres(wl["set_off"], wl["set_items"], seeds)
        so, si = subset_rows(wl["set_off"], wl["set_items"], rows)
        lab, inter, uni = assign_jaccard(so, si, coff, cit)
        res.update(centre_off=coff, centre_items=cit, labels=lab, inter=inter, union=uni)
    else:
        attrs = hetero_attrs(res["numeric_buckets"], wl["cat"])
        m = modes(attrs, seeds)
        lab, mt = assign_cat(attrs[rows], m)
        res.update(attrs=attrs, modes=m, labels=lab, matches=mt)
    return res
