"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer results (codes, bucket ids, members, seeds, labels) must be
bit-exact; SSE and radius within 1e-6 relative of the oracle's FP64 values.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

RTOL_SSE = 1e-6


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    return geek


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


def check_buckets(got, ref, codes_ref=None):
    assert np.array_equal(got["n_buckets"], ref.n_buckets)
    assert np.array_equal(got["obj_bucket"].cpu().numpy(), ref.obj_bucket)
    assert np.array_equal(got["bucket_off"].cpu().numpy(), ref.boff)
    assert np.array_equal(got["members"].cpu().numpy(), ref.bmem)
    if codes_ref is not None:
        assert np.array_equal(got["codes"].cpu().numpy(), codes_ref.astype(np.int32))


def run_dense(G, ctx, wl, proj=0):
    cfg = wl["cfg"]
    x = G._dev(wl["x"])
    bk = ctx.hash(ctx.dense(x), cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=wl["w"], proj=proj)
    return x, bk


@pytest.mark.parametrize("over", [dict(), dict(n=1), dict(n=4097), dict(n=20000, silk=dict(delta=1))])
def test_dense_c1_full_pipeline(G, ctx, over):
    """Small dense workload: codes, buckets, seeds, labels and SSE."""
    wl = synth.make(synth.config("c1", **over))
    cfg = wl["cfg"]
    x, bk = run_dense(G, ctx, wl)
    ref = oracle.run_workload(wl)
    check_buckets(bk.copy_out(), ref["buckets"], ref["codes"])
    seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
    assert seeds.n_multiset == ref["seeds"].n_multiset
    assert seeds.sets() == ref["seeds"].sets()
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    centres = torch.empty((max(seeds.k, 1), cfg.d), dtype=torch.float64, device="cuda")
    st = ctx.assign(ctx.dense(x), bk, seeds, labels, centers=centres)
    torch.cuda.synchronize()
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    if seeds.k:
        assert np.array_equal(centres[: seeds.k].cpu().numpy(), ref["centres"])  # bit-exact FP64
        sse = float(np.sum(ref["dist"]))
        assert abs(st.sse - sse) <= RTOL_SSE * sse
        assert abs(st.radius_max - np.sqrt(ref["dist"].max())) <= RTOL_SSE * np.sqrt(ref["dist"].max())


@pytest.mark.parametrize("mode", ["all", "first"])
@pytest.mark.parametrize("delta", [2, 1])
def test_silk_minhash_functions_that_repeat_values(G, ctx, mode, delta):
    """SILK hashes that repeat values on neighbouring ids (multipliers near
    2^31).  "all": every function of the even tables repeats, so one-object
    virtual buckets share signatures and take the general grouping path;
    "first": one function per table stays injective on the ids (the
    one-object path) while first components collide everywhere.  Seeds
    equal the oracle's."""
    wl = synth.make(synth.config("c1"))
    cfg = wl["cfg"]
    sp = dict(synth.silk_params_slow(wl["silk"], mode), delta=delta)
    x, bk = run_dense(G, ctx, wl)
    _, ref_b = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    ref_s = oracle.silk_on(ref_b, sp)
    assert ref_s.n_multiset > 0
    seeds = ctx.silk(bk, **G.silk_args(sp))
    assert seeds.n_multiset == ref_s.n_multiset
    assert seeds.sets() == ref_s.sets()


def test_dense_c2_shape_hash_and_assign(G, ctx):
    """The 10M x 128 workload's shape at n = 60,000 (several tiles, ragged
    tail): E2LSH K=6, L=16 codes and buckets, then assignment to the planted
    centres in both fast precisions."""
    wl = synth.make(synth.config("c2", n=60_001, n_comp=600))
    cfg = wl["cfg"]
    x, bk = run_dense(G, ctx, wl)
    codes, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    check_buckets(bk.copy_out(), ref, codes)
    assert bk.n_flagged > 0  # the window does flag elements at this scale
    assert 0 <= bk.n_flagged_fp64 <= bk.n_flagged
    c = wl["centres"].astype(np.float64)
    lab_ref, dist_ref = oracle.assign_dense(wl["x"], c)
    for prec in (G.PREC_FP32, G.PREC_BF16, G.PREC_BF16X3):
        labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
        st = ctx.assign_centers(ctx.dense(x), G._dev(c), labels, precision=prec)
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), lab_ref), prec
        assert abs(st.sse - dist_ref.sum()) <= RTOL_SSE * dist_ref.sum()


def test_srp_codes_and_buckets(G, ctx):
    wl = synth.make(synth.config("c1", n=9000))
    cfg = wl["cfg"]
    x, bk = run_dense(G, ctx, wl, proj=G.PROJ_SRP)
    bits, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L, proj="srp")
    check_buckets(bk.copy_out(), ref, bits)


@pytest.mark.parametrize("d", [33, 7])
def test_odd_dimension_codes_and_buckets(G, ctx, d):
    """d not a multiple of 4: the projection stages rows without 16-byte
    copies; codes, buckets and the tcgen05 assignment stay exact."""
    wl = synth.make(synth.config("c1", n=6001, d=d))
    cfg = wl["cfg"]
    x, bk = run_dense(G, ctx, wl)
    codes, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    check_buckets(bk.copy_out(), ref, codes)
    c = wl["centres"].astype(np.float64)
    lab_ref, _ = oracle.assign_dense(wl["x"], c)
    for prec in (G.PREC_BF16, G.PREC_BF16X3):
        labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
        ctx.assign_centers(ctx.dense(x), G._dev(c), labels, precision=prec)
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), lab_ref), prec


def test_assign_near_ties_are_exact(G, ctx):
    """Duplicated and nearly duplicated centres force the FP64 decision:
    exact ties must go to the smaller index."""
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((5000, 32)) * 3).astype(np.float32)
    c = rng.standard_normal((300, 32)) * 3
    c[150:] = c[:150]                      # exact duplicates
    c[100:150] += 1e-9                     # near duplicates
    lab_ref, _ = oracle.assign_dense(x, c)
    for prec in (G.PREC_FP32, G.PREC_BF16, G.PREC_BF16X3):
        labels = torch.empty(5000, dtype=torch.int32, device="cuda")
        st = ctx.assign_centers(ctx.dense(G._dev(x)), G._dev(c), labels, precision=prec)
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), lab_ref)
        assert st.n_recheck_rows > 0
        # exact ties cannot be settled by any window: they reach FP64
        assert 0 < st.n_fp64_rows <= st.n_recheck_rows


def test_host_memory_path(G, ctx):
    """The same call with host buffers (the library stages them)."""
    wl = synth.make(synth.config("c1", n=5000))
    cfg = wl["cfg"]
    c = wl["centres"].astype(np.float64)
    lab_ref, _ = oracle.assign_dense(wl["x"], c)
    labels = np.empty(cfg.n, dtype=np.int32)
    ctx.assign_centers(ctx.dense(wl["x"], host=True), c, labels)
    assert np.array_equal(labels, lab_ref)


def test_resident_upload_shared_by_hash_and_assign(G, ctx):
    """geek_data_upload: one device copy of host data serves hash, SILK and
    the assignment; the handle is reused by smaller and larger uploads."""
    res = ctx.resident()
    for n in (5000, 1200, 9000):
        wl = synth.make(synth.config("c1", n=n))
        cfg = wl["cfg"]
        xh = np.ascontiguousarray(wl["x"])
        dv = res.upload(ctx.dense(xh, host=True))
        assert dv.c.mem == G.MEM_DEVICE and dv.c.n == n and dv.c.d == cfg.d
        bk = ctx.hash(dv, cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=wl["w"])
        ref = oracle.run_workload(wl)
        check_buckets(bk.copy_out(), ref["buckets"], ref["codes"].astype(np.int32))
        seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
        assert seeds.sets() == ref["seeds"].sets()
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assign(dv, bk, seeds, labels, precision=G.PREC_BF16)
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    wl = synth.make(synth.config("c3", n=3001, n_base=50))
    cfg = wl["cfg"]
    dv = res.upload(ctx.sets(wl["set_off"], wl["set_items"].astype(np.uint32), host=True))
    bk = ctx.hash(dv, cfg.K, cfg.L, mh_a=G._dev(wl["mh_a"]), mh_b=G._dev(wl["mh_b"]))
    ref = oracle.run_workload(wl)
    check_buckets(bk.copy_out(), ref["buckets"], ref["codes"].view(np.int32))
    with pytest.raises(G.GeekError) as e:
        res.upload(ctx.dense(G._dev(np.zeros((4, 4), np.float32))))  # device data: nothing to upload
    assert e.value.status == G.ERR_INVALID


def test_invalid_arguments_are_reported(G, ctx):
    wl = synth.make(synth.config("c1", n=100))
    x = G._dev(wl["x"])
    with pytest.raises(G.GeekError) as e:
        ctx.hash(ctx.dense(x), 0, 8, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=4.0)
    assert e.value.status == G.ERR_INVALID
    with pytest.raises(G.GeekError):
        ctx.hash(ctx.dense(x), 4, 8, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=-1.0)


@pytest.mark.parametrize("over", [dict(n=20_000, n_base=200), dict(n=3001, n_base=50, silk=dict(delta=3))])
def test_sets_c3_shape_pipeline(G, ctx, over):
    """Sparse sets: MinHash K=4, L=32 (128-bit table keys), SILK, majority
    centres and exact Jaccard assignment."""
    wl = synth.make(synth.config("c3", **over))
    cfg = wl["cfg"]
    off = G._dev(wl["set_off"])
    items = G._dev(wl["set_items"].astype(np.int32))
    data = ctx.sets(off, items)
    bk = ctx.hash(data, cfg.K, cfg.L, mh_a=G._dev(wl["mh_a"]), mh_b=G._dev(wl["mh_b"]))
    ref = oracle.run_workload(wl)
    assert bk.key_bits_max == 128
    got = bk.copy_out()
    check_buckets(got, ref["buckets"], ref["codes"].view(np.int32))
    seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
    assert seeds.sets() == ref["seeds"].sets()
    assert seeds.k > 0
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    _, cen = ctx.assign_ex(data, bk, seeds, labels)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    check_sparse_centres(cen, ref)


def check_sparse_centres(cen, ref):
    """Majority item sets of the seeds (Sect. 3.3), element by element."""
    assert np.array_equal(cen["item_off"].cpu().numpy(), ref["centre_off"])
    assert np.array_equal(cen["items"].cpu().numpy().view(np.uint32), ref["centre_items"])


def check_modes(cen, ref, wl):
    """Per-attribute modes (Sect. 3.3): numeric attributes as canonical
    ranks, categorical ones as tokens (= offset of the attribute + value)."""
    tok_off = (wl["tokens"][0].astype(np.int64) - wl["cat"][0].astype(np.int64))
    L = ref["attrs"].shape[1] - tok_off.size
    m = cen["modes"].cpu().numpy()
    assert m.shape == ref["modes"].shape
    assert np.array_equal(m[:, :L], ref["modes"][:, :L])
    assert np.array_equal(m[:, L:] - tok_off[None, :], ref["modes"][:, L:])


@pytest.mark.parametrize("over", [dict(n=20_000, n_comp=100), dict(n=777, n_comp=20, silk=dict(delta=1))])
def test_hetero_c4_shape_pipeline(G, ctx, over):
    """Heterogeneous rows: E2LSH codes of the numeric part concatenated with
    MinHash of the tokens (Alg. 2), SILK, modes and categorical assignment."""
    wl = synth.make(synth.config("c4", **over))
    cfg = wl["cfg"]
    x = G._dev(wl["x"])
    tok = G._dev(wl["tokens"].astype(np.int32))
    data = ctx.hetero(x, tok)
    bk = ctx.hash(data, cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=wl["w"],
                  mh_a=G._dev(wl["mh_a"]), mh_b=G._dev(wl["mh_b"]), Kc=cfg.Kc)
    ref = oracle.run_workload(wl)
    check_buckets(bk.copy_out(), ref["buckets"], ref["codes"])
    seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
    assert seeds.sets() == ref["seeds"].sets()
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    _, cen = ctx.assign_ex(data, bk, seeds, labels)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    if seeds.k:
        check_modes(cen, ref, wl)


# ------------------------------------------- Alg. 1 (QALSH, even split) --
def qalsh_buckets(G, ctx, x, a, t):
    m = a.shape[0]
    bk = ctx.hash(ctx.dense(G._dev(x)), 1, m, a=G._dev(a), proj=G.PROJ_QALSH, t=t)
    torch.cuda.synchronize()
    return bk


def check_alg1(got, ref):
    assert np.array_equal(got["n_buckets"], ref.n_buckets)
    assert np.array_equal(got["obj_bucket"].cpu().numpy(), ref.obj_bucket)
    assert np.array_equal(got["bucket_off"].cpu().numpy(), ref.boff)
    assert np.array_equal(got["members"].cpu().numpy(), ref.bmem)


@pytest.mark.parametrize("n,m,t", [(20000, 8, 7), (20000, 8, 1), (6001, 5, 6001), (30001, 12, 300), (777, 3, 50)])
def test_alg1_buckets_exact(G, ctx, n, m, t):
    """Alg. 1: the FP32 order is fixed near every cut with FP64 values, so
    the parts equal the oracle's exact split (sizes, members, ids)."""
    wl = synth.make(synth.config("c1", n=n))
    x, a = wl["x"], wl["a"][:m]
    bk = qalsh_buckets(G, ctx, x, a, t)
    _, ref = oracle.transform_alg1(x, a, t)
    check_alg1(bk.copy_out(), ref)


def test_alg1_ties_and_near_ties(G, ctx):
    """Duplicated rows (exact ties, decided by id), rows a few ulps apart
    across the cuts, and zero rows (+0 and -0 projections)."""
    rng = np.random.default_rng(17)
    n, d, m, t = 5000, 16, 6, 40
    x = rng.standard_normal((n, d)).astype(np.float32)
    x[1000:1400] = x[5]                      # 400 identical rows
    x[2000:2300] = 0.0                       # projections exactly 0
    x[2300:2310] = -0.0
    base = x[300].copy()
    for i in range(3000, 3600):              # rows within a few ulps of each other
        x[i] = np.nextafter(base, np.float32(np.inf)) if i % 2 else base
    a = rng.standard_normal((m, d)).astype(np.float32)
    bk = qalsh_buckets(G, ctx, x, a, t)
    _, ref = oracle.transform_alg1(x, a, t)
    check_alg1(bk.copy_out(), ref)


@pytest.mark.parametrize("t", [400, 100])
def test_alg1_feeds_silk_and_assignment(G, ctx, t):
    """Alg. 1 buckets through SILK seeding and the one-pass assignment
    (t = 100: buckets of 120 objects, so the SILK signatures take the
    thread-per-set kernel; t = 400: 30 objects, the thread per (set, table))."""
    wl = synth.make(synth.config("c1", n=12000))
    x, a = wl["x"], wl["a"][:16]
    bk = qalsh_buckets(G, ctx, x, a, t)
    _, ref_b = oracle.transform_alg1(x, a, t)
    seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
    ref_s = oracle.silk_on(ref_b, wl["silk"])
    assert seeds.sets() == ref_s.sets()
    if seeds.k:
        labels = torch.empty(x.shape[0], dtype=torch.int32, device="cuda")
        ctx.assign(ctx.dense(G._dev(x)), bk, seeds, labels, precision=G.PREC_BF16)
        torch.cuda.synchronize()
        c = oracle.centroids(x, ref_s)
        lab_ref, _ = oracle.assign_dense(x, c)
        assert np.array_equal(labels.cpu().numpy(), lab_ref)


def test_alg1_invalid(G, ctx):
    wl = synth.make(synth.config("c1", n=100))
    x = G._dev(wl["x"])
    for K, t in ((2, 10), (1, 0), (1, 101)):
        with pytest.raises(G.GeekError) as e:
            ctx.hash(ctx.dense(x), K, 4, a=G._dev(wl["a"][:4 * K]), proj=G.PROJ_QALSH, t=t)
        assert e.value.status == G.ERR_INVALID


def test_assign_all_centres_in_the_window(G, ctx):
    """Every centre nearly equal: each flagged row has every centre of a tile
    inside its window (128 x 64 pairs per tile, several rounds of the FP64
    decision's queue), with exact duplicates for the index tie-break."""
    rng = np.random.default_rng(17)
    n, d, k = 3000, 32, 200
    x = (rng.standard_normal((n, d)) * 2).astype(np.float32)
    base = rng.standard_normal(d) * 2
    c = base[None, :] + rng.standard_normal((k, d)) * 1e-9
    c[100:] = c[:100]  # exact duplicates
    lab_ref, _ = oracle.assign_dense(x, c)
    for prec in (G.PREC_FP32, G.PREC_BF16, G.PREC_BF16X3):
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        st = ctx.assign_centers(ctx.dense(G._dev(x)), G._dev(c), labels, precision=prec)
        torch.cuda.synchronize()
        if prec != G.PREC_FP32:  # the tensor-core forms end in the tiled FP64 decision
            assert st.n_fp64_rows > n // 2
        assert np.array_equal(labels.cpu().numpy(), lab_ref)


def _w_bf16x3(xn, cmax, d):
    """The split-BF16 assignment's half-window (the kernel's rigorous bound,
    per-product accumulation model), evaluated in float64."""
    ub = 2.0 ** -8
    xc, c2 = xn * cmax, cmax * cmax
    e = (6 * ub * ub * (1 + ub) * xc + 2.0 ** -24 * c2
         + (3 * d + 19) * 2.0 ** -21 * (2 * xc * (1 + 4 * ub) + c2 * (1 + 2 * ub)))
    s = xn + cmax
    return 1.01 * (e + (d + 3) * 2.0 ** -53 * s * s)


def test_assign_just_outside_the_window(G, ctx):
    """Rows placed 1.05-1.6 windows from a tie between the two centres of a
    pair, with |x| |c| ~ 6e5 against distance gaps of a few hundred (heavy
    cancellation in |c|^2 - 2 x.c): the split-BF16 tensor-core pass settles
    most of them alone, so an accumulation error beyond the modelled bound
    would show as a wrong label."""
    rng = np.random.default_rng(31)
    n, d, P, off = 20000, 64, 50, 100.0
    B = rng.standard_normal((P, d)) * 30 + off
    u = rng.standard_normal((P, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = np.empty((2 * P, d))
    c[0::2], c[1::2] = B + u, B - u
    cmax = np.sqrt((c.astype(np.float32).astype(np.float64) ** 2).sum(1).max()) * (1 + 1e-5)
    p = rng.integers(0, P, n)
    x = B[p] + rng.standard_normal((n, d))
    g = rng.uniform(1.05, 1.6, n)
    for _ in range(4):  # the window grows with |x|: place, then re-place
        W = 2 * _w_bf16x3(np.sqrt((x ** 2).sum(1)) * (1 + 1e-3), cmax, d) * (1 + 1e-6)
        gap = ((x - c[2 * p + 1]) ** 2).sum(1) - ((x - c[2 * p]) ** 2).sum(1)
        x += ((g * W - gap) / 4.0)[:, None] * u[p]  # |c1 - c2| = 2: the gap moves 4 per unit along u
    x = x.astype(np.float32)
    lab_ref, _ = oracle.assign_dense(x, c)
    assert np.array_equal(lab_ref, 2 * p)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    st = ctx.assign_centers(ctx.dense(G._dev(x)), G._dev(c), labels, precision=G.PREC_BF16X3)
    torch.cuda.synchronize()
    assert np.array_equal(labels.cpu().numpy(), lab_ref)
    assert st.n_recheck_rows < n // 2


def test_cluster_radius(G, ctx):
    """Per-cluster radius (Sect. 4.1): sqrt of the largest FP64 distance of a
    member to its centre, within 1e-6 relative of the oracle's; 0 for a
    cluster with no member; a label of -1 is skipped."""
    wl = synth.make(synth.config("c1", n=20_000))
    x = wl["x"]
    c = np.concatenate([wl["centres"].astype(np.float64), np.full((1, x.shape[1]), 1e5)])  # an empty cluster
    lab, dist = oracle.assign_dense(x, c)
    lab = lab.astype(np.int32)
    lab[::97] = -1
    k = c.shape[0]
    ref = np.zeros(k)
    for j in range(k):
        m = lab == j
        if m.any():
            ref[j] = np.sqrt(dist[m].max())
    radius = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
    ctx.cluster_radius(ctx.dense(G._dev(x)), G._dev(c), G._dev(lab), radius)
    torch.cuda.synchronize()
    got = radius.cpu().numpy()
    assert got[-1] == 0.0
    assert np.all(np.abs(got - ref) <= RTOL_SSE * ref)


# ------------------------------------- extra passes of assignment (Sect. 5) --
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_refine_passes_exact(G, ctx, prec):
    """geek_refine: each pass's centres (FP64 means in ascending id) and
    labels bit-exact against the oracle; a centre nobody is nearest to keeps
    its value."""
    P = G.PREC_BF16 if prec == "bf16" else G.PREC_FP32
    wl = synth.make(synth.config("c1", n=9000))
    x = wl["x"]
    c0 = wl["centres"].astype(np.float64)
    c0 = np.concatenate([c0, np.full((1, x.shape[1]), 1e5)])  # an empty cluster
    lab0, _ = oracle.assign_dense(x, c0)
    xd, cd = G._dev(x), G._dev(c0)
    labels = G._dev(lab0.astype(np.int32))
    st = ctx.refine(ctx.dense(xd), cd, labels, 3, precision=P)
    torch.cuda.synchronize()
    lab_ref, c_ref, dist = oracle.refine_passes(x, c0, lab0, 3)
    assert np.array_equal(labels.cpu().numpy(), lab_ref)
    assert np.array_equal(cd.cpu().numpy(), c_ref)
    assert np.array_equal(c_ref[-1], c0[-1])
    sse = float(dist.sum())
    assert abs(st.sse - sse) <= 1e-6 * sse


@pytest.mark.parametrize("d", [70, 128])
def test_refine_ragged_slices_and_large_clusters(G, ctx, d):
    """The centre update works on 32-coordinate slices of a centre: d = 70
    leaves a ragged slice of 6; one cluster holds most rows (its member list
    spans many 32-row batches and ends mid-batch); rows come from a strided
    view (row pitch d + 10)."""
    rng = np.random.default_rng(11 + d)
    n, k = 7001, 6
    full = rng.standard_normal((n, d + 10)).astype(np.float32)
    full[: n - 300, :d] += 4.0  # the big cluster
    x = full[:, :d]
    c0 = rng.standard_normal((k, d)) * 2
    c0[0] += 4.0
    lab0, _ = oracle.assign_dense(np.ascontiguousarray(x), c0)
    xt = G._dev(full)[:, :d]
    cd = G._dev(c0)
    labels = G._dev(lab0.astype(np.int32))
    ctx.refine(ctx.dense(xt), cd, labels, 2, precision=G.PREC_BF16)
    torch.cuda.synchronize()
    lab_ref, c_ref, _ = oracle.refine_passes(np.ascontiguousarray(x), c0, lab0, 2)
    assert np.bincount(lab_ref, minlength=k).max() > 5000
    assert np.array_equal(labels.cpu().numpy(), lab_ref)
    assert np.array_equal(cd.cpu().numpy(), c_ref)


def _hard_sum_rows(n, rng):
    """Rows whose coordinates make the centre update's running FP64 sums
    change binade often, hit exact half-ulp ties, span FP32 exponents from
    -149 to 20 (subnormals included), or hold signed zeros."""
    d = 96
    x = np.zeros((n, d), dtype=np.float32)
    x[:, 0:16] = rng.standard_normal((n, 16))                        # random walks around 0
    x[:, 16:24] = np.where(np.arange(n)[:, None] % 2 == 0, 1.0, 2.0 ** -53)  # ties at s near 1
    x[:, 24:32] = np.where(np.arange(n)[:, None] % 3 == 0, 3.0, -(2.0 ** -52) * 3)
    e = rng.integers(-149, 21, (n, 24))
    x[:, 32:56] = (rng.uniform(1, 2, (n, 24)) * rng.choice([-1.0, 1.0], (n, 24)) * np.exp2(e.astype(np.float64)))
    x[:, 56:64] = np.where(rng.random((n, 8)) < 0.5, 0.0, -0.0)       # signed zeros
    x[:, 64:72] = rng.uniform(-1e-38, 1e-38, (n, 8))                   # around the FP32 subnormal range
    x[:, 72:96] = rng.normal(20.0, 1.0, (n, 24))                       # linear growth
    return x


def test_refine_centre_update_hard_sums(G, ctx):
    """The centre update's integer steps and their FP64 fallback: one live
    cluster of rows built to change binade, tie and underflow; its FP64 mean
    (ascending id) must equal the oracle's bit for bit."""
    rng = np.random.default_rng(23)
    n = 5003
    x = _hard_sum_rows(n, rng)
    c0 = np.zeros((2, x.shape[1]))
    c0[1] = 1e6  # nobody's nearest: stays unchanged
    lab0 = np.zeros(n, dtype=np.int32)
    cd = G._dev(c0)
    labels = G._dev(lab0)
    ctx.refine(ctx.dense(G._dev(x)), cd, labels, 1, precision=G.PREC_FP32)
    torch.cuda.synchronize()
    _, c_ref, _ = oracle.refine_passes(x, c0, lab0, 1)
    got = cd.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), c_ref.view(np.uint64))


def test_refine_invalid_labels(G, ctx):
    wl = synth.make(synth.config("c1", n=500))
    c = G._dev(wl["centres"].astype(np.float64))
    labels = torch.full((500,), c.shape[0], dtype=torch.int32, device="cuda")  # out of range
    with pytest.raises(G.GeekError) as e:
        ctx.refine(ctx.dense(G._dev(wl["x"])), c, labels, 1)
    assert e.value.status == G.ERR_INVALID


# -------------------------------------------- DOPH step of Alg. 3 (sets) --
@pytest.mark.parametrize("Dp", [64, 400])
def test_sets_doph_transform(G, ctx, Dp):
    """Alg. 3 with DOPH: the reduced tokens' MinHash values and the buckets
    bit-exact against the oracle (sets larger and smaller than Dp, an empty
    set)."""
    wl = synth.make(synth.config("c3", n=4000, n_base=80))
    cfg = wl["cfg"]
    off = np.concatenate([wl["set_off"], [wl["set_off"][-1]]]).astype(np.int64)  # + one empty set
    items = wl["set_items"].astype(np.uint32)
    rng = np.random.default_rng(Dp)
    Ap, Bp = int(rng.integers(1, 1 << 62)) * 2 + 1, int(rng.integers(0, 1 << 62))
    data = ctx.sets(G._dev(off), G._dev(items.astype(np.int32)))
    bk = ctx.hash(data, cfg.K, cfg.L, mh_a=G._dev(wl["mh_a"]), mh_b=G._dev(wl["mh_b"]), doph_bins=Dp,
                  doph_a=Ap, doph_b=Bp)
    _, mh, ref = oracle.transform_sparse_doph(off, items, Dp, Ap, Bp, wl["mh_a"], wl["mh_b"], cfg.K, cfg.L)
    got = bk.copy_out()
    assert np.array_equal(got["codes"].cpu().numpy().view(np.uint32), mh)
    check_buckets(got, ref)


@pytest.mark.parametrize("Dp", [64, 400])
def test_sets_doph_pipeline(G, ctx, Dp):
    """Alg. 3 with DOPH through SILK and the assignment (Sect. 3.3): seeds,
    the per-dimension modes of the reduced tokens and every label against
    the oracle."""
    wl = synth.make(synth.config("c3", n=6000, n_base=60, silk=dict(delta=4)))
    cfg = wl["cfg"]
    rng = np.random.default_rng(Dp + 1)
    Ap, Bp = int(rng.integers(1, 1 << 62)) * 2 + 1, int(rng.integers(0, 1 << 62))
    wl["doph"] = dict(bins=Dp, a=Ap, b=Bp)
    data = ctx.sets(G._dev(wl["set_off"]), G._dev(wl["set_items"].astype(np.int32)))
    bk = ctx.hash(data, cfg.K, cfg.L, mh_a=G._dev(wl["mh_a"]), mh_b=G._dev(wl["mh_b"]), doph_bins=Dp,
                  doph_a=Ap, doph_b=Bp)
    seeds = ctx.silk(bk, **G.silk_args(wl["silk"]))
    ref = oracle.run_workload(wl)
    assert seeds.sets() == ref["seeds"].sets()
    assert seeds.k > 0
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    _, cen = ctx.assign_ex(data, bk, seeds, labels)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    assert np.array_equal(cen["modes"].cpu().numpy(), ref["modes"])
