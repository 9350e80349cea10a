"""GPU parity of the batched form: many dense instances of uneven n, d and
seed count in one geek_batch (one projection launch, one persistent tcgen05
assignment launch, CUDA graphs, autotuned centre tiles).

Every instance's codes, bucket ids, seeds, centroids and labels must be
bit-exact against the FP64 oracle run on that instance alone; SSE and radius
within 1e-6 relative.  The batch must also agree with the single-instance
C ABI run instance by instance, for every centre-tile width.
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


def dev_instance(G, I):
    sp = I["silk"]
    return dict(x=G._dev(I["x"]), a=G._dev(I["a"]), b=G._dev(I["b"]), w=I["w"], mh_a=G._dev(sp["mh_a"]),
                mh_b=G._dev(sp["mh_b"]), dd_a=G._dev(sp["dd_a"]), dd_b=G._dev(sp["dd_b"]))


def make_batch(G, ctx, insts, tile_n=0, precision=None):
    cfg = insts[0]["cfg"]
    s = insts[0]["silk"]
    dev = [dev_instance(G, I) for I in insts]
    prec = G.PREC_AUTO if precision is None else precision
    return G.Batch(ctx, dev, cfg.K, cfg.L, s["Ks"], s["Ls"], s["delta"], tile_n=tile_n, precision=prec), dev


def run_batch(b):
    labels = torch.empty(max(int(b.row_off[-1]), 1), dtype=torch.int32, device="cuda")
    b.run(labels)
    torch.cuda.synchronize()
    return labels.cpu().numpy()[: int(b.row_off[-1])]


def small_batch():
    insts = synth.batch_instances(count=9, n_range=(300, 6000), comp_range=(10, 60), seed=synth.ROOT_SEED + 51)
    # a one-object instance: no bin has two buckets, so no seed and label -1
    tiny = synth.batch_instances(count=1, n_range=(1, 1), comp_range=(10, 10), seed=synth.ROOT_SEED + 52)[0]
    insts.insert(4, tiny)
    return insts


def test_batch_matches_oracle_per_instance(G, ctx):
    insts = small_batch()
    assert len({I["x"].shape[1] for I in insts}) >= 2  # uneven d
    b, _ = make_batch(G, ctx, insts)
    labels = run_batch(b)
    got = b.copy_out()
    info = b.info()
    assert info["count"] == len(insts)
    for i, I in enumerate(insts):
        ref = oracle.run_workload(dict(cfg=I["cfg"], x=I["x"], a=I["a"], b=I["b"], w=I["w"], silk=I["silk"]))
        g = got[i]
        r0, r1 = b.row_off[i], b.row_off[i + 1]
        assert np.array_equal(g["codes"], ref["codes"].astype(np.int32)), i
        assert np.array_equal(g["obj_bucket"], ref["buckets"].obj_bucket), i
        assert g["seeds"] == ref["seeds"].sets(), i
        assert np.array_equal(labels[r0:r1], ref["labels"]), i
        if g["k"]:
            assert np.array_equal(g["centres"], ref["centres"]), i  # bit-exact FP64
            sse = float(np.sum(ref["dist"]))
            assert abs(g["sse"] - sse) <= RTOL_SSE * sse, i
            rm = float(np.sqrt(ref["dist"].max()))
            assert abs(g["radius_max"] - rm) <= RTOL_SSE * rm, i
        else:
            assert (labels[r0:r1] == -1).all()
    assert got[4]["k"] == 0 and labels[b.row_off[4]] == -1
    assert sum(g["k"] for g in got) > 0


@pytest.mark.parametrize("mode", ["all", "first"])
def test_batch_minhash_functions_that_repeat_values(G, ctx, mode):
    """SILK hashes that repeat values on neighbouring ids (multipliers near
    2^31): "all" gives one instance repeating functions in every even table
    (one-object virtual buckets share signatures: the general grouping path
    for the whole batch), "first" makes every instance's first function of
    every table repeat (the one-object path stays on).  Seeds equal the
    oracle's instance by instance."""
    insts = small_batch()
    for i, I in enumerate(insts):
        if mode == "first" or i == 2:
            I["silk"] = synth.silk_params_slow(I["silk"], mode, seed=synth.ROOT_SEED + 70 + i)
    b, _ = make_batch(G, ctx, insts)
    run_batch(b)
    got = b.copy_out()
    for i, I in enumerate(insts):
        cfg = I["cfg"]
        _, ref_b = oracle.hash_dense(I["x"], I["a"], I["b"], I["w"], cfg.K, cfg.L)
        assert got[i]["seeds"] == oracle.silk_on(ref_b, I["silk"]).sets(), i


def test_batch_tiles_replay_and_sequential_agree(G, ctx):
    insts = synth.batch_instances(count=14, n_range=(2000, 40000), comp_range=(10, 400), seed=synth.ROOT_SEED + 53)
    b, dev = make_batch(G, ctx, insts)
    lab = run_batch(b)
    st = b.instance_stats()
    info1 = b.info()
    assert set(st["tile_n"].tolist()) <= {64, 128, 256}
    assert info1["graph_captures"] >= 2 and info1["graph_launches"] >= 2
    # replay: the same graphs, the same results
    lab2 = run_batch(b)
    info2 = b.info()
    assert np.array_equal(lab, lab2)
    assert info2["graph_captures"] == info1["graph_captures"]
    assert info2["graph_launches"] == info1["graph_launches"] + 2
    assert set(st["precision"].tolist()) <= {G.PREC_BF16, G.PREC_BF16X3}
    # every forced tile width and precision gives the same labels
    rows = {}
    for prec, tn in ((G.PREC_BF16, 64), (G.PREC_BF16, 128), (G.PREC_BF16, 256), (G.PREC_BF16X3, 64),
                     (G.PREC_BF16X3, 128)):
        bt, _ = make_batch(G, ctx, insts, tile_n=tn, precision=prec)
        assert np.array_equal(run_batch(bt), lab), (prec, tn)
        s2 = bt.instance_stats()
        assert set(s2["precision"].tolist()) == {prec}
        ds = np.array([I["x"].shape[1] for I in insts])
        cap = np.where(ds <= 64, 128, 64) if prec == G.PREC_BF16X3 else 256
        assert (s2["tile_n"] == np.minimum(tn, cap)).all(), (prec, tn)
        rows[prec] = bt.info()["n_recheck_rows"]
    # the split-BF16 window is ~100x narrower: fewer rows need the FP64 decision
    assert rows[G.PREC_BF16X3] <= rows[G.PREC_BF16]
    # the single-instance C ABI, instance by instance
    got = b.copy_out()
    for i, (I, D) in enumerate(zip(insts, dev)):
        cfg = I["cfg"]
        bk = ctx.hash(ctx.dense(D["x"]), cfg.K, cfg.L, a=D["a"], b=D["b"], w=D["w"])
        seeds = ctx.silk(bk, **G.silk_args(I["silk"]))
        assert seeds.sets() == got[i]["seeds"], i
        labels = torch.empty(cfg.n, dtype=torch.int32, device="cuda")
        s = ctx.assign(ctx.dense(D["x"]), bk, seeds, labels, precision=G.PREC_BF16)
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), lab[b.row_off[i]:b.row_off[i + 1]]), i
        if seeds.k:
            assert abs(s.sse - st["sse"][i]) <= RTOL_SSE * s.sse, i
    # one small instance against the oracle as well
    j = int(np.argmin([I["cfg"].n for I in insts]))
    I = insts[j]
    ref = oracle.run_workload(dict(cfg=I["cfg"], x=I["x"], a=I["a"], b=I["b"], w=I["w"], silk=I["silk"]))
    assert np.array_equal(lab[b.row_off[j]:b.row_off[j + 1]], ref["labels"])


def test_batch_invalid_arguments(G, ctx):
    insts = synth.batch_instances(count=2, n_range=(100, 200), comp_range=(10, 20), seed=synth.ROOT_SEED + 54)
    with pytest.raises(G.GeekError) as e:
        make_batch(G, ctx, insts, tile_n=100)
    assert e.value.status == G.ERR_INVALID
    wide = synth.batch_instances(count=1, n_range=(100, 100), d_choices=(130,), comp_range=(10, 10),
                                 seed=synth.ROOT_SEED + 55)
    with pytest.raises(G.GeekError) as e:
        make_batch(G, ctx, wide)
    assert e.value.status == G.ERR_UNSUPPORTED
