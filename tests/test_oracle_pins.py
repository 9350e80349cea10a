"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks one oracle function against an independent statement of
what the paper fixes: exact rational arithmetic, Python big integers, dict /
Counter brute force on tiny inputs, the worked Example 2 (Sect. 3.2), the
MinHash collision law (Eq. 2), and invariants of SILK (Alg. 4).
"""
import json
import math
import os
import random
from collections import Counter, defaultdict
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
M64 = 1 << 64


def hbig(A, B, x):
    return ((int(A) * int(x) + int(B)) % M64) >> 32


# ----------------------------------------------------------------- E2LSH --
def exact_codes(x, a, b, w):
    n, d = x.shape
    F = a.shape[0]
    out = np.empty((n, F), dtype=np.int64)
    gap = np.empty((n, F))
    for i in range(n):
        for f in range(F):
            v = sum(Fraction(float(a[f, j])) * Fraction(float(x[i, j])) for j in range(d))
            t = (v + Fraction(float(b[f]))) / Fraction(w)
            fl = math.floor(t)
            out[i, f] = fl
            gap[i, f] = float(min(t - fl, fl + 1 - t))
    return out, gap


def test_e2lsh_matches_exact_rational_floor(orc):
    rng = np.random.default_rng(1)
    n, d, F = 40, 7, 5  # d != F so a transposed operand cannot pass
    x = (rng.standard_normal((n, d)) * 20).astype(np.float32)
    a = rng.standard_normal((F, d)).astype(np.float32)
    b = (rng.random(F) * 4).astype(np.float32)
    got = orc.e2lsh(x, a, b, 4.0)
    want, gap = exact_codes(x, a, b, 4.0)
    near = gap < 1e-9
    assert near.sum() == 0  # random inputs: no exact-boundary ambiguity
    assert np.array_equal(got, want)
    # a non-power-of-two width exercises the rounded division
    got3 = orc.e2lsh(x, a, b, 3.0)
    want3, gap3 = exact_codes(x, a, b, 3.0)
    assert np.array_equal(got3[gap3 > 1e-9], want3[gap3 > 1e-9])


def test_e2lsh_handcrafted_boundaries(orc):
    # a.x + b lands exactly on / just beside multiples of w, and negative
    # values check floor (not truncation toward zero)
    a = np.array([[0.5, 0.0], [1.0, -1.0]], dtype=np.float32)
    b = np.array([0.0, 0.5], dtype=np.float32)
    x = np.array([[8.0, 3.0], [-2.0, 0.0], [7.999999, 1.0], [-8.0, 4.0], [0.0, 0.5]], dtype=np.float32)
    got = orc.e2lsh(x, a, b, 4.0)
    want, _ = exact_codes(x, a, b, 4.0)
    assert np.array_equal(got, want)
    assert got[0, 0] == 1 and got[1, 0] == -1 and got[2, 0] == 0 and got[3, 0] == -1
    # property: floor(t) <= t < floor(t) + 1 for every element
    rng = np.random.default_rng(2)
    xs = (rng.standard_normal((20, 3)) * 9).astype(np.float32)
    aa = rng.standard_normal((4, 3)).astype(np.float32)
    bb = (rng.random(4) * 4).astype(np.float32)
    c = orc.e2lsh(xs, aa, bb, 4.0)
    t = (xs.astype(np.float64) @ aa.T.astype(np.float64) + bb) / 4.0
    assert np.all(c <= t + 1e-9) and np.all(t < c + 1 + 1e-9)


def test_e2lsh_overflow_is_reported(orc):
    x = np.array([[3e38]], dtype=np.float32)
    a = np.array([[1.0]], dtype=np.float32)
    with pytest.raises(RuntimeError):
        orc.e2lsh(x, a, np.zeros(1, np.float32), 4.0)


def test_srp_matches_exact_sign(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((30, 6)).astype(np.float32)
    a = rng.standard_normal((9, 6)).astype(np.float32)
    x[0] = 0.0  # a.x == 0 exactly counts as >= 0
    got = orc.srp(x, a)
    for i in range(30):
        for f in range(9):
            v = sum(Fraction(float(a[f, j])) * Fraction(float(x[i, j])) for j in range(6))
            assert got[i, f] == (1 if v >= 0 else 0)


# --------------------------------------------------- DOPH (Alg. 3 step) --
def test_doph_hand_worked_bins():
    """pi(v) = v (A = 2^32, B = 0), 4 bins = the top two bits of v, offset =
    the low 30 bits times 4.  Worked by hand from the definition."""
    import oracle
    S = [0x40000005, 0x40000003, 0xC0000001]
    tok = oracle.doph(np.array([0, 3, 4], dtype=np.int64), np.array(S + [2], dtype=np.uint32), 4, 1 << 32, 0)
    want0 = [(0 << 48) | (1 << 32) | 0xC,   # bin 0 empty: borrows bin 1 at distance 1
             (1 << 48) | (0 << 32) | 0xC,   # min(0x14, 0xC)
             (2 << 48) | (1 << 32) | 0x4,   # bin 2 empty: borrows bin 3
             (3 << 48) | (0 << 32) | 0x4]
    assert [int(v) for v in tok[0]] == want0
    # one item in bin 0: bins 1..3 borrow it across the wrap-around
    want1 = [(0 << 48) | 8, (1 << 48) | (3 << 32) | 8, (2 << 48) | (2 << 32) | 8, (3 << 48) | (1 << 32) | 8]
    assert [int(v) for v in tok[1]] == want1


def test_doph_collision_rate_is_jaccard():
    """Rotation-densified OPH is an LSH for resemblance: for every bin,
    Pr[token(S1) == token(S2)] = |S1 n S2| / |S1 u S2| over random pi."""
    import oracle
    rng = np.random.default_rng(44)
    pool = rng.choice(1 << 31, size=100, replace=False).astype(np.uint32)
    S1, S2 = pool[:80], pool[20:100]  # |n| = 60, |u| = 100
    J = 0.6
    off = np.array([0, 80, 160], dtype=np.int64)
    items = np.concatenate([S1, S2])
    trials, Dp = 1500, 6
    hits = np.zeros(Dp)
    for _ in range(trials):
        A, B = int(rng.integers(1, 1 << 63)) * 2 + 1, int(rng.integers(0, 1 << 63))
        t = oracle.doph(off, items, Dp, A, B)
        hits += (t[0] == t[1])
    rate = hits / trials
    sd = math.sqrt(J * (1 - J) / trials)
    assert np.all(np.abs(rate - J) < 4.5 * sd), rate


def test_minhash_rows64_big_integers():
    import oracle
    rng = np.random.default_rng(45)
    tok = rng.integers(0, 1 << 63, size=(7, 5), dtype=np.uint64) * 2 + 1
    A = rng.integers(0, 1 << 63, size=4, dtype=np.uint64)
    B = rng.integers(0, 1 << 63, size=4, dtype=np.uint64)
    got = oracle.minhash_rows64(tok, A, B)
    for i in range(7):
        for f in range(4):
            assert got[i, f] == min(((int(A[f]) * int(x) + int(B[f])) % M64) >> 32 for x in tok[i])


# ------------------------------------------------- Alg. 1 (QALSH split) --
def exact_alg1(x, a, t):
    """Alg. 1 by hand: exact rational projections, objects sorted by (value,
    id), the sorted list cut at floor(b n / t)."""
    n, d = x.shape
    ob = np.empty((a.shape[0], n), dtype=np.int64)
    for f in range(a.shape[0]):
        v = [sum(Fraction(float(a[f, j])) * Fraction(float(x[i, j])) for j in range(d)) for i in range(n)]
        order = sorted(range(n), key=lambda i: (v[i], i))
        cuts = [(b * n) // t for b in range(t)] + [n]
        for b in range(t):
            for pos in range(cuts[b], cuts[b + 1]):
                ob[f, order[pos]] = b
    return ob


@pytest.mark.parametrize("n,t", [(61, 7), (40, 1), (23, 23), (50, 3)])
def test_alg1_matches_exact_rational_split(orc, n, t):
    rng = np.random.default_rng(n * 31 + t)
    x = rng.standard_normal((n, 5)).astype(np.float32)
    a = rng.standard_normal((3, 5)).astype(np.float32)
    x[7 % n] = x[3 % n]  # two identical objects: equal values, id order decides
    s, B = orc.transform_alg1(x, a, t)
    assert np.array_equal(B.obj_bucket, exact_alg1(x, a, t))
    # every table is a partition into t parts of the even sizes
    want = np.diff((np.arange(t + 1) * n) // t)
    for f in range(3):
        assert np.array_equal(np.bincount(B.obj_bucket[f], minlength=t), want)
        # part b's values never exceed part b + 1's
        for b in range(t - 1):
            lo, hi = s[B.obj_bucket[f] == b, f], s[B.obj_bucket[f] == b + 1, f]
            if lo.size and hi.size:
                assert lo.max() <= hi.min()
    assert B.NB == 3 * t
    # members ascending inside each bucket, offsets at f * n + floor(b n / t)
    for g in range(B.NB):
        mem = B.bmem[B.boff[g]:B.boff[g + 1]]
        assert np.all(np.diff(mem) > 0)
    assert B.boff[1] == (n // t if t > 1 else n)


def test_alg1_ties_follow_ids(orc):
    # all objects equal: every projection ties, so the parts are id ranges
    x = np.ones((10, 4), dtype=np.float32)
    a = np.random.default_rng(2).standard_normal((2, 4)).astype(np.float32)
    _, B = orc.transform_alg1(x, a, 3)
    assert B.obj_bucket.tolist() == [[0, 0, 0, 1, 1, 1, 2, 2, 2, 2]] * 2


# --------------------------------------------------------------- MinHash --
def test_hash32_against_big_integers(orc):
    rng = random.Random(4)
    for _ in range(2000):
        A, B, x = rng.getrandbits(64), rng.getrandbits(64), rng.getrandbits(32)
        assert orc.hash32(A, B, x) == hbig(A, B, x)
    assert orc.hash32(M64 - 1, M64 - 1, 0xFFFFFFFF) == hbig(M64 - 1, M64 - 1, 0xFFFFFFFF)


def test_minhash_explicit_minima(orc):
    rng = np.random.default_rng(5)
    sets = [sorted(rng.choice(1 << 20, size=s, replace=False).tolist()) for s in [1, 2, 5, 33, 64, 100]]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    items = np.array([i for s in sets for i in s], np.uint32)
    A = rng.integers(0, 2**63, 11, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    B = rng.integers(0, 2**63, 11, dtype=np.uint64)
    got = orc.minhash_csr(off, items, A, B)
    for i, s in enumerate(sets):
        for f in range(11):
            assert got[i, f] == min(hbig(A[f], B[f], v) for v in s)
    # the empty set (undefined in the paper) maps to 0xFFFFFFFF
    e = orc.minhash_csr(np.array([0, 0], np.int64), np.zeros(0, np.uint32), A[:1], B[:1])
    assert e[0, 0] == 0xFFFFFFFF


def test_minhash_collision_rate_equals_jaccard(orc):
    """Eq. 2: Pr[h(A) = h(B)] = J(A, B); 20,000 independent hashes, 4 sigma."""
    rng = np.random.default_rng(6)
    univ = rng.choice(1 << 20, size=150, replace=False)
    A_set = np.sort(univ[:90])
    B_set = np.sort(univ[45:135])  # |A n B| = 45, |A u B| = 135 -> J = 1/3
    J = 45 / 135
    T = 20000
    ca = rng.integers(0, np.iinfo(np.uint64).max, T, dtype=np.uint64, endpoint=True)
    cb = rng.integers(0, np.iinfo(np.uint64).max, T, dtype=np.uint64, endpoint=True)
    off = np.array([0, 90, 180], np.int64)
    mh = orc.minhash_csr(off, np.concatenate([A_set, B_set]).astype(np.uint32), ca, cb)
    rate = np.mean(mh[0] == mh[1])
    sigma = math.sqrt(J * (1 - J) / T)
    assert abs(rate - J) < 4 * sigma, (rate, J)


# -------------------------------------------------------------- grouping --
def test_sort_rows_is_stable_lexicographic(orc):
    rng = np.random.default_rng(7)
    for n in [1, 17, 70000]:
        keys = rng.integers(-3, 3, size=(n, 3)).astype(np.int64)
        perm = np.empty(n, np.int32)
        orc.lib().orc_sort_rows(n, 3, orc._p(keys), orc._p(perm))
        want = np.lexsort((np.arange(n), keys[:, 2], keys[:, 1], keys[:, 0]))
        assert np.array_equal(perm, want)


def test_group_against_dict(orc):
    rng = np.random.default_rng(8)
    L, n, W = 3, 500, 4
    keys = rng.integers(-2, 2, size=(L, n, W)).astype(np.int64)
    bk = orc.group(keys)
    for l in range(L):
        groups = defaultdict(list)
        for i in range(n):
            groups[tuple(keys[l, i])].append(i)
        ordered = sorted(groups)
        assert bk.n_buckets[l] == len(ordered)
        for r, kk in enumerate(ordered):
            g = bk.table_base[l] + r
            mem = bk.bmem[bk.boff[g]:bk.boff[g + 1]].tolist()
            assert mem == groups[kk]  # ascending ids inside the bucket
            for i in groups[kk]:
                assert bk.obj_bucket[l, i] == r


# ------------------------------------------------------------------ SILK --
def test_example2_vote_forced_bins(orc):
    """Sect. 3.2, Example 2: majority voting on the printed bins of T1."""
    g = json.load(open(os.path.join(GOLD, "example2_silk.json")))
    names = sorted(g["buckets"], key=lambda s: int(s[1:]))
    buckets = [g["buckets"][nm] for nm in names]
    idx = {nm: i for i, nm in enumerate(names)}
    bins = [[idx[b] for b in g["bins_T1"][k]] for k in ["Bin1", "Bin2", "Bin3"]]
    got = orc.vote_bins(bins, buckets, g["delta"])
    assert got[0] == tuple(g["expected_C_shared_T1"]["Bin1"])
    assert got[1] == tuple(g["expected_C_shared_T1"]["Bin2"])
    assert got[2] == ()  # |Bin3| <= 1: ignored
    # the strict "more than half" rule: an object in exactly half is dropped
    assert orc.vote_bins([[0, 1]], [[1, 2], [2, 3]], 1) == [(2,)]
    # delta filter
    assert orc.vote_bins([[0, 1]], [[1, 2], [1, 2]], 3) == [()]


def test_example2_dedup_forced_bins(orc):
    """Sect. 3.2, Example 2: the multiset from both tables deduplicates to the
    four printed seeds when the two copies of {x1,x2,x4} share a bin."""
    g = json.load(open(os.path.join(GOLD, "example2_silk.json")))
    ms = [tuple(s) for s in g["multiset_after_both_tables"]]
    bins = [[0, 2], [1], [3], [4]]
    got = orc.dedup_bins(ms, bins, g["delta"])
    assert sorted(got) == sorted(tuple(s) for s in g["expected_final_seeds"])
    assert got == sorted(got)  # canonical order
    # a bin of several sets whose vote is below delta keeps its smallest member
    assert orc.dedup_bins([(1, 2), (3, 4)], [[0, 1]], 1) == [(1, 2)]


def silk_brute(buckets, Ks, Ls, delta, A, B, dA, dB):
    """Alg. 4 restated with dicts and Counters on tiny inputs."""
    def sig(s, a, b):
        return tuple(min(hbig(a[k], b[k], i) for i in s) for k in range(len(a)))
    C = []
    for t in range(Ls):
        a, b = A[t * Ks:(t + 1) * Ks], B[t * Ks:(t + 1) * Ks]
        bins = defaultdict(list)
        for bk in buckets:
            bins[sig(bk, a, b)].append(bk)
        for mem in bins.values():
            if len(mem) <= 1:
                continue
            cnt = Counter(i for bk in mem for i in bk)
            cs = tuple(sorted(i for i, c in cnt.items() if 2 * c > len(mem)))
            if len(cs) >= delta:
                C.append(cs)
    bins = defaultdict(list)
    for s in C:
        bins[sig(s, dA, dB)].append(s)
    D = []
    for mem in bins.values():
        if len(mem) == 1:
            D.append(mem[0])
            continue
        cnt = Counter(i for s in mem for i in s)
        vs = tuple(sorted(i for i, c in cnt.items() if 2 * c > len(mem)))
        D.append(vs if len(vs) >= delta else min(mem))
    return sorted(set(D)), len(C)


def small_hash_coeffs(rng, m, modulus_bits=3):
    # coefficients chosen so that collisions (and hence non-trivial bins)
    # are frequent on tiny inputs: A*x+B with tiny A keeps the high word small
    A = rng.integers(0, 1 << modulus_bits, m, dtype=np.uint64) << np.uint64(29)
    B = rng.integers(0, 1 << 40, m, dtype=np.uint64)
    return A, B


@pytest.mark.parametrize("seed", range(12))
def test_silk_against_brute_force(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = 30
    buckets = []
    for _ in range(40):
        s = int(rng.integers(1, 7))
        buckets.append(tuple(sorted(rng.choice(n, size=s, replace=False).tolist())))
    Ks, Ls, delta = int(rng.integers(1, 3)), int(rng.integers(1, 5)), int(rng.integers(1, 3))
    A, B = small_hash_coeffs(rng, Ks * Ls)
    dA, dB = small_hash_coeffs(rng, Ks)
    boff = np.zeros(len(buckets) + 1, np.int64)
    boff[1:] = np.cumsum([len(b) for b in buckets])
    bmem = np.array([i for b in buckets for i in b], np.int32)
    got = orc.silk(boff, bmem, Ks, Ls, delta, A, B, dA, dB)
    want, nC = silk_brute(buckets, Ks, Ls, delta, A, B, dA, dB)
    assert got.sets() == want
    assert got.n_multiset == nC
    # bucket order must not matter (bins are sets of buckets)
    perm = rng.permutation(len(buckets))
    pb = [buckets[i] for i in perm]
    boff2 = np.zeros(len(pb) + 1, np.int64)
    boff2[1:] = np.cumsum([len(b) for b in pb])
    bmem2 = np.array([i for b in pb for i in b], np.int32)
    assert orc.silk(boff2, bmem2, Ks, Ls, delta, A, B, dA, dB).sets() == want


def test_silk_more_tables_more_candidates(orc):
    """Example 3: more SILK tables can only add C_shared sets to the multiset
    (the first tables' hashes are shared)."""
    import synth
    wl = synth.make(synth.config("c1", n=4000))
    codes, bk = orc.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], 4, 8)
    sp = wl["silk"]
    prev = -1
    for Ls in [1, 5, 10, 20]:
        s = orc.silk(bk.boff, bk.bmem, sp["Ks"], Ls, sp["delta"], sp["mh_a"][: Ls * sp["Ks"]],
                     sp["mh_b"][: Ls * sp["Ks"]], sp["dd_a"], sp["dd_b"])
        assert s.n_multiset >= prev
        prev = s.n_multiset
        for j in range(s.k):  # canonical: ascending members, distinct seeds
            m = s.ids[s.off[j]:s.off[j + 1]]
            assert m.size >= 1 and np.all(np.diff(m) > 0)
        assert s.sets() == sorted(set(s.sets()))


# ------------------------------------------------------------ assignment --
def test_centroids_exact_mean_within_one_ulp(orc):
    rng = np.random.default_rng(9)
    x = (rng.standard_normal((60, 5)) * 13).astype(np.float32)
    sets = [sorted(rng.choice(60, size=s, replace=False).tolist()) for s in [1, 2, 3, 7, 31, 60]]
    seeds = orc.Seeds(np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64),
                      np.array([i for s in sets for i in s], np.int32), len(sets))
    c = orc.centroids(x, seeds)
    for j, s in enumerate(sets):
        for t in range(5):
            exact = sum(Fraction(float(x[i, t])) for i in s) / len(s)
            assert abs(Fraction(c[j, t]) - exact) <= Fraction(np.spacing(abs(c[j, t])))


def test_assign_dense_exhaustive_exact(orc):
    rng = np.random.default_rng(10)
    x = (rng.standard_normal((120, 4)) * 5).astype(np.float32)
    c = rng.standard_normal((9, 4)) * 5
    c[7] = c[2]  # exact tie: the smaller index must win
    lab, dist = orc.assign_dense(x, c)
    for i in range(120):
        D = [sum((Fraction(float(x[i, t])) - Fraction(c[j, t])) ** 2 for t in range(4)) for j in range(9)]
        m = min(D)
        assert lab[i] == D.index(m)
        assert abs(dist[i] - float(m)) <= 1e-12 * float(m) + 1e-300
    assert not np.any(lab == 7)
    lab0, _ = orc.assign_dense(x, np.zeros((0, 4)))
    assert np.all(lab0 == -1)


# ------------------------------------------ extra passes (Sect. 5) --
def test_refine_blobs_reach_exact_means(orc):
    """Three far-apart blobs and centres that start inside the wrong blobs'
    neighbourhood: one pass moves every centre to the exact rational mean
    of its blob (within 1 ulp), and the labels become the blobs."""
    rng = np.random.default_rng(21)
    blobs = [np.array([0.0, 0.0, 0.0]), np.array([100.0, 0.0, 0.0]), np.array([0.0, 100.0, 0.0])]
    x = np.concatenate([(b + rng.standard_normal((40, 3))).astype(np.float32) for b in blobs])
    truth = np.repeat(np.arange(3), 40)
    c0 = np.array([[10.0, 0, 0], [80.0, 5, 0], [5.0, 90, 0]])
    lab0, _ = orc.assign_dense(x, c0)
    assert np.array_equal(lab0, truth)
    lab, c, dist = orc.refine_passes(x, c0, lab0, 1)
    assert np.array_equal(lab, truth)
    for j in range(3):
        pts = x[truth == j]
        for t in range(3):
            exact = sum(Fraction(float(v)) for v in pts[:, t]) / len(pts)
            assert abs(c[j, t] - float(exact)) <= abs(np.spacing(float(exact)))
    # a fixed point: another pass changes nothing
    lab2, c2, _ = orc.refine_passes(x, c, lab, 1)
    assert np.array_equal(lab2, lab) and np.array_equal(c2, c)


def test_refine_sse_never_increases_and_empty_centres_stay(orc):
    rng = np.random.default_rng(22)
    x = (rng.standard_normal((400, 5)) * 3).astype(np.float32)
    c = rng.standard_normal((12, 5)) * 3
    c[11] = 1e6  # no object is nearest to it: it keeps its value
    lab, dist = orc.assign_dense(x, c)
    sse = float(dist.sum())
    for _ in range(4):
        lab, c_new, dist = orc.refine_passes(x, c, lab, 1)
        assert np.array_equal(c_new[11], c[11])
        assert float(dist.sum()) <= sse * (1 + 1e-12)
        sse, c = float(dist.sum()), c_new


def test_modes_and_categorical_assignment(orc):
    rng = np.random.default_rng(11)
    n, A = 80, 6
    attrs = rng.integers(0, 4, size=(n, A)).astype(np.int64)
    sets = [sorted(rng.choice(n, size=s, replace=False).tolist()) for s in [1, 2, 4, 9, 20]]
    seeds = orc.Seeds(np.concatenate([[0], np.cumsum([len(s) for s in sets])]).astype(np.int64),
                      np.array([i for s in sets for i in s], np.int32), len(sets))
    m = orc.modes(attrs, seeds)
    for j, s in enumerate(sets):
        for a in range(A):
            cnt = Counter(int(attrs[i, a]) for i in s)
            top = max(cnt.values())
            assert m[j, a] == min(v for v, c in cnt.items() if c == top)
    lab, mt = orc.assign_cat(attrs, m)
    for i in range(n):
        scores = [int(np.sum(attrs[i] == m[j])) for j in range(len(sets))]
        assert mt[i] == max(scores) and lab[i] == scores.index(max(scores))


def test_sparse_centres_and_jaccard(orc):
    rng = np.random.default_rng(12)
    n = 50
    sets = [sorted(rng.choice(40, size=int(rng.integers(1, 12)), replace=False).tolist()) for _ in range(n)]
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    items = np.array([i for s in sets for i in s], np.uint32)
    seed_sets = [sorted(rng.choice(n, size=s, replace=False).tolist()) for s in [1, 3, 4, 8]]
    seeds = orc.Seeds(np.concatenate([[0], np.cumsum([len(s) for s in seed_sets])]).astype(np.int64),
                      np.array([i for s in seed_sets for i in s], np.int32), len(seed_sets))
    coff, cit = orc.sparse_centres(off, items, seeds)
    cents = []
    for j, ss in enumerate(seed_sets):
        cnt = Counter(v for i in ss for v in sets[i])
        want = sorted(v for v, c in cnt.items() if 2 * c > len(ss))
        assert cit[coff[j]:coff[j + 1]].tolist() == want
        cents.append(set(want))
    cents.append(set())  # an empty centre: similarity 0
    coff2 = np.concatenate([coff, [coff[-1]]])
    lab, inter, uni = orc.assign_jaccard(off, items, coff2, cit)
    for i, s in enumerate(sets):
        J = [Fraction(len(set(s) & c), len(set(s) | c)) if (s or c) else Fraction(0) for c in cents]
        assert lab[i] == J.index(max(J))
        assert Fraction(int(inter[i]), int(uni[i])) == max(J)


# ------------------------------------------------- heterogeneous rows (Alg. 2) --
def test_hetero_keys_and_attrs_from_the_formula(orc):
    """Alg. 2 reading: table l's key is (E2LSH codes of functions l*K .. l*K+K-1
    on the numeric part) followed by (MinHash values of functions
    l*Kc .. l*Kc+Kc-1 on the token set {offset_j + v_j}); the unified
    attributes of Sect. 3.3 are, per table, the rank of the numeric-only tuple
    among the table's distinct numeric tuples, then the raw categorical
    values.  Rebuilt here with exact rationals, big integers and dicts; K != Kc
    and L != n_cat so a swapped slice or attribute order cannot pass."""
    rng = np.random.default_rng(21)
    n, d, K, L, Kc, n_cat, w = 60, 3, 2, 3, 3, 4, 4.0
    cards = [3, 5, 2, 7]
    x = (rng.standard_normal((n, d)) * 3).astype(np.float32)
    x[n // 2:] = x[: n - n // 2]                 # repeated numeric parts share buckets
    a = rng.standard_normal((K * L, d)).astype(np.float32)
    b = (rng.random(K * L) * 4).astype(np.float32)
    cat = np.stack([rng.integers(0, c, size=n) for c in cards], axis=1).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(cards)[:-1]])
    tokens = (cat + offs[None, :]).astype(np.uint32)
    A = rng.integers(0, 1 << 63, size=Kc * L, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    B = rng.integers(0, 1 << 63, size=Kc * L, dtype=np.uint64)
    codes, mh, bk, nbk = orc.hash_hetero(x, tokens, a, b, w, K, L, A, B, Kc)

    want_codes, _ = exact_codes(x, a, b, w)
    assert np.array_equal(codes, want_codes)
    want_mh = np.array([[min(hbig(A[f], B[f], t) for t in tokens[i]) for f in range(Kc * L)] for i in range(n)])
    assert np.array_equal(mh, want_mh)

    attrs = orc.hetero_attrs(nbk, cat)
    assert attrs.shape == (n, L + n_cat)
    for l in range(L):
        full = [tuple(int(v) for v in want_codes[i, l * K:(l + 1) * K]) +
                tuple(int(v) for v in want_mh[i, l * Kc:(l + 1) * Kc]) for i in range(n)]
        num = [tuple(int(v) for v in want_codes[i, l * K:(l + 1) * K]) for i in range(n)]
        for keys, got in ((full, bk), (num, nbk)):
            rank = {k: r for r, k in enumerate(sorted(set(keys)))}
            assert got.n_buckets[l] == len(rank)
            assert [int(v) for v in got.obj_bucket[l]] == [rank[k] for k in keys]
            members = defaultdict(list)
            for i, k in enumerate(keys):
                members[rank[k]].append(i)
            base = int(got.table_base[l])
            for r in range(len(rank)):
                lo, hi = got.boff[base + r], got.boff[base + r + 1]
                assert got.bmem[lo:hi].tolist() == members[r]
        num_rank = {k: r for r, k in enumerate(sorted(set(num)))}
        assert [int(v) for v in attrs[:, l]] == [num_rank[k] for k in num]
    assert np.array_equal(attrs[:, L:], cat)
    # the split is a real concatenation: some numeric buckets are cut by MinHash
    assert any(bk.n_buckets[l] > nbk.n_buckets[l] for l in range(L))


def test_doph_modes_and_assignment(orc):
    """Sect. 3.3 for sets reduced by DOPH: the centre is the per-dimension
    mode of the members' tokens; the label maximises the dimensions equal to
    it (1 - Jaccard of D' tokens against D' tokens), ties to the smallest."""
    rng = np.random.default_rng(31)
    n, Dp = 60, 5
    sets = [sorted(rng.choice(40, size=int(rng.integers(0, 9)), replace=False).tolist()) for _ in range(n)]
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    items = np.array([i for s in sets for i in s], np.uint32)
    Ap, Bp = 0x9E3779B97F4A7C15, 12345
    tok = orc.doph(off, items, Dp, Ap, Bp)
    seed_sets = [sorted(rng.choice(n, size=s, replace=False).tolist()) for s in [1, 2, 5, 9, 14]]
    seeds = orc.Seeds(np.concatenate([[0], np.cumsum([len(s) for s in seed_sets])]).astype(np.int64),
                      np.array([i for s in seed_sets for i in s], np.int32), len(seed_sets))
    m = orc.doph_modes(tok, seeds)
    for j, ss in enumerate(seed_sets):
        for b in range(Dp):
            cnt = Counter(int(tok[i, b]) for i in ss)
            top = max(cnt.values())
            assert int(m[j, b]) == min(v for v, c in cnt.items() if c == top)
            assert int(m[j, b]) >> 48 == b  # the mode of dimension b is a dimension-b token
    lab, mt = orc.assign_doph(tok, m)
    for i in range(n):
        sc = [sum(int(tok[i, b]) == int(m[j, b]) for b in range(Dp)) for j in range(len(seed_sets))]
        assert mt[i] == max(sc) and lab[i] == sc.index(max(sc))
        # the same label by exact Jaccard of the D' tokens
        J = [Fraction(len(set(tok[i].tolist()) & set(m[j].astype(np.uint64).tolist())),
                      len(set(tok[i].tolist()) | set(m[j].astype(np.uint64).tolist()))) for j in range(len(seed_sets))]
        assert lab[i] == J.index(max(J))
