"""Full-size parity at every workload's stated size, against the oracle.

* 10M x 128 dense points, in the configuration bench.py times (E2LSH K=6,
  L=16, w=4 on the tensor cores, and on the FP32 path; SILK Ks=3, Ls=10,
  delta=10; assignment to the 20,000 planted centres in both fast
  precisions): every code, every canonical bucket id, the SILK seed set,
  and the labels of 4,096 sampled points.
* 2M sparse sets (MinHash K=4, L=32; Jaccard assignment): every MinHash
  value, every bucket id, the seed list, every majority-item centre, and
  4,096 sampled labels.
* 2M heterogeneous rows (E2LSH K=4, L=8 on 20 numeric attributes, MinHash
  Kc=2 on 10 categorical ones): every code, every bucket id, the seed list,
  every mode, and 4,096 sampled labels.
* The 256-instance batch (33.75M rows): per instance every code and bucket
  id, the seed list, the FP64 centroids, and 512 sampled labels.

Every comparison is exact, element by element; the oracle computes each
sampled label exhaustively over all centres."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_c2_full_size():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    wl = synth.make(synth.config("c2"))
    cfg = wl["cfg"]
    ctx = geek.Context(0)
    x = geek._dev(wl["x"])
    data = ctx.dense(x)
    bk = ctx.hash(data, cfg.K, cfg.L, a=geek._dev(wl["a"]), b=geek._dev(wl["b"]), w=wl["w"],
                  precision=geek.PREC_BF16X3)
    seeds = ctx.silk(bk, **geek.silk_args(wl["silk"]))
    bk32 = ctx.hash(data, cfg.K, cfg.L, a=geek._dev(wl["a"]), b=geek._dev(wl["b"]), w=wl["w"])
    g_codes32 = bk32.copy_out()["codes"].cpu().numpy()
    del bk32
    centres = wl["centres"].astype(np.float64)
    labs = {}
    for prec in (geek.PREC_BF16, geek.PREC_FP32):
        labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
        ctx.assign_centers(data, geek._dev(centres), labels, precision=prec)
        labs[prec] = labels.cpu().numpy()
    got = bk.copy_out()
    g_codes = got["codes"].cpu().numpy()
    g_ob = got["obj_bucket"].cpu().numpy()
    g_seeds = seeds.sets()
    del got, bk, x
    torch.cuda.empty_cache()

    codes = oracle.e2lsh(wl["x"], wl["a"], wl["b"], wl["w"])
    assert np.array_equal(g_codes, codes)        # tcgen05 projection
    assert np.array_equal(g_codes32, codes)      # FP32 SIMT projection
    del g_codes, g_codes32
    ref = oracle.group(oracle.table_keys(codes, cfg.L, cfg.K))
    assert np.array_equal(g_ob, ref.obj_bucket)
    del g_ob
    ref_seeds = oracle.silk_on(ref, wl["silk"])
    assert g_seeds == ref_seeds.sets()

    rows = np.sort(np.random.default_rng(7).choice(cfg.n, 4096, replace=False))
    lab_ref, _ = oracle.assign_dense(wl["x"][rows], centres)
    for prec, lab in labs.items():
        assert np.array_equal(lab[rows], lab_ref), prec


def test_alg1_full_size_sampled_tables():
    """Alg. 1 at the bench's size and configuration (10M x 128, m = 40
    QALSH tables, t = 20,000 buckets): every bucket id of 4 sampled tables
    against the oracle's exact split, and the even bucket sizes of all 40."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    wl = synth.make(synth.config("c2"))
    n = wl["cfg"].n
    m, t = 40, 20000
    a = np.ascontiguousarray(wl["a"][:m])
    ctx = geek.Context(0)
    bk = ctx.hash(ctx.dense(geek._dev(wl["x"])), 1, m, a=geek._dev(a), proj=geek.PROJ_QALSH, t=t)
    got = bk.copy_out()
    ob = got["obj_bucket"].cpu().numpy()
    boff = got["bucket_off"].cpu().numpy()
    del got, bk
    torch.cuda.empty_cache()
    sizes = np.diff(boff)
    want = np.diff((np.arange(t + 1) * n) // t)
    assert np.array_equal(sizes, np.tile(want, m))
    tables = np.random.default_rng(11).choice(m, 4, replace=False)
    s = oracle.qalsh(wl["x"], a[tables])
    for q, f in enumerate(tables):
        assert np.array_equal(ob[f], oracle.split_even(s[:, q], t)), f


def _sample(n, m=4096, seed=7):
    return np.sort(np.random.default_rng(seed).choice(n, min(m, n), replace=False))


def test_c3_sets_full_size():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    wl = synth.make(synth.config("c3"))
    cfg = wl["cfg"]
    ctx = geek.Context(0)
    data = ctx.sets(geek._dev(wl["set_off"]), geek._dev(wl["set_items"].astype(np.int32)))
    bk = ctx.hash(data, cfg.K, cfg.L, mh_a=geek._dev(wl["mh_a"]), mh_b=geek._dev(wl["mh_b"]))
    seeds = ctx.silk(bk, **geek.silk_args(wl["silk"]))
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    _, cen = ctx.assign_ex(data, bk, seeds, labels)
    got = bk.copy_out()
    g_mh = got["codes"].cpu().numpy().view(np.uint32)
    g_ob = got["obj_bucket"].cpu().numpy()
    g_seeds = seeds.sets()
    g_coff, g_cit = cen["item_off"].cpu().numpy(), cen["items"].cpu().numpy().view(np.uint32)
    g_lab = labels.cpu().numpy()
    del got, bk, data, cen, labels
    torch.cuda.empty_cache()

    rows = _sample(cfg.n)
    ref = oracle.run_workload(wl, assign_rows=rows)
    assert np.array_equal(g_mh, ref["codes"])
    assert np.array_equal(g_ob, ref["buckets"].obj_bucket)
    assert len(g_seeds) == ref["seeds"].k > 0
    assert g_seeds == ref["seeds"].sets()
    assert np.array_equal(g_coff, ref["centre_off"])
    assert np.array_equal(g_cit, ref["centre_items"])
    assert np.array_equal(g_lab[rows], ref["labels"])


def test_c4_hetero_full_size():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    wl = synth.make(synth.config("c4"))
    cfg = wl["cfg"]
    ctx = geek.Context(0)
    data = ctx.hetero(geek._dev(wl["x"]), geek._dev(wl["tokens"].astype(np.int32)))
    bk = ctx.hash(data, cfg.K, cfg.L, a=geek._dev(wl["a"]), b=geek._dev(wl["b"]), w=wl["w"],
                  mh_a=geek._dev(wl["mh_a"]), mh_b=geek._dev(wl["mh_b"]), Kc=cfg.Kc)
    seeds = ctx.silk(bk, **geek.silk_args(wl["silk"]))
    labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
    _, cen = ctx.assign_ex(data, bk, seeds, labels)
    got = bk.copy_out()
    g_codes = got["codes"].cpu().numpy()
    g_ob = got["obj_bucket"].cpu().numpy()
    g_seeds = seeds.sets()
    g_modes = cen["modes"].cpu().numpy()
    g_lab = labels.cpu().numpy()
    del got, bk, data, cen, labels
    torch.cuda.empty_cache()

    rows = _sample(cfg.n)
    ref = oracle.run_workload(wl, assign_rows=rows)
    assert np.array_equal(g_codes, ref["codes"])
    assert np.array_equal(g_ob, ref["buckets"].obj_bucket)
    assert len(g_seeds) == ref["seeds"].k > 0
    assert g_seeds == ref["seeds"].sets()
    # modes: numeric attributes as canonical ranks, categorical ones as tokens
    tok_off = wl["tokens"][0].astype(np.int64) - wl["cat"][0].astype(np.int64)
    L = cfg.L
    assert np.array_equal(g_modes[:, :L], ref["modes"][:, :L])
    assert np.array_equal(g_modes[:, L:] - tok_off[None, :], ref["modes"][:, L:])
    assert np.array_equal(g_lab[rows], ref["labels"])


def test_c5_batch_full_size():
    """All 256 instances in one batch; the oracle runs instance by instance
    in a pool of host processes while the results are compared."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    import oracle_pool
    insts = synth.batch_instances(threads=8)
    ctx = geek.Context(0)
    cfg = insts[0]["cfg"]
    s = insts[0]["silk"]
    dev = [dict(x=geek._dev(I["x"]), a=geek._dev(I["a"]), b=geek._dev(I["b"]), w=I["w"],
                mh_a=geek._dev(I["silk"]["mh_a"]), mh_b=geek._dev(I["silk"]["mh_b"]),
                dd_a=geek._dev(I["silk"]["dd_a"]), dd_b=geek._dev(I["silk"]["dd_b"])) for I in insts]
    b = geek.Batch(ctx, dev, cfg.K, cfg.L, s["Ks"], s["Ls"], s["delta"])
    N = int(b.row_off[-1])
    labels = torch.empty(N, dtype=torch.int32, device="cuda")
    b.run(labels)
    torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    got = b.copy_out()
    row_off = np.array(b.row_off)
    ns = [I["cfg"].n for I in insts]
    del b, dev, labels, insts
    torch.cuda.empty_cache()

    seen = 0
    for ref in oracle_pool.run(np.argsort(ns)[::-1]):
        i = ref["i"]
        g = got[i]
        assert np.array_equal(g["codes"], ref["codes"]), i
        assert np.array_equal(g["obj_bucket"], ref["obj_bucket"]), i
        assert g["seeds"] == ref["seeds"], i
        if g["k"]:
            assert np.array_equal(g["centres"], ref["centres"]), i  # bit-exact FP64
        assert np.array_equal(lab[row_off[i]:row_off[i + 1]][ref["rows"]], ref["labels"]), i
        seen += 1
    assert seen == 256
    assert sum(g["k"] for g in got) > 0


def test_alg1_silk_assign_full_size():
    """The paper's own pipeline on the 10M x 128 points: Alg. 1 (m = 40
    QALSH tables, t = 5,000 even buckets each), SILK on those buckets
    (Ks = 2, Ls = 20, delta = 10), FP64 centroids of the seeds and the
    one-pass assignment to them.  The seed list and every centroid are
    compared exactly, and 4,096 sampled labels in both fast precisions."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    wl = synth.make(synth.config("c2"))
    n, d = wl["x"].shape
    m, t = synth.ALG1["m"], synth.ALG1["t"]
    sp = synth.alg1_silk_params()
    a = np.ascontiguousarray(wl["a"][:m])
    ctx = geek.Context(0)
    data = ctx.dense(geek._dev(wl["x"]))
    bk = ctx.hash(data, 1, m, a=geek._dev(a), proj=geek.PROJ_QALSH, t=t)
    seeds = ctx.silk(bk, **geek.silk_args(sp))
    g_seeds = seeds.sets()
    labs = {}
    cen = torch.empty((max(seeds.k, 1), d), dtype=torch.float64, device="cuda")
    for prec in (geek.PREC_BF16, geek.PREC_FP32):
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assign(data, bk, seeds, labels, centers=cen, precision=prec)
        labs[prec] = labels.cpu().numpy()
    g_cen = cen[: seeds.k].cpu().numpy()
    del bk, data, cen
    torch.cuda.empty_cache()

    _, ref_bk = oracle.transform_alg1(wl["x"], a, t)
    ref_seeds = oracle.silk_on(ref_bk, sp)
    del ref_bk
    assert len(g_seeds) == ref_seeds.k > 0
    assert g_seeds == ref_seeds.sets()
    ref_c = oracle.centroids(wl["x"], ref_seeds)
    assert np.array_equal(g_cen, ref_c)  # bit-exact FP64
    rows = _sample(n)
    lab_ref, _ = oracle.assign_dense(wl["x"][rows], ref_c)
    for prec, lab in labs.items():
        assert np.array_equal(lab[rows], lab_ref), prec
