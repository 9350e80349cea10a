"""Full-size parity on the 10M x 128 workload, in the configuration bench.py
times (E2LSH K=6, L=16, w=4; SILK Ks=3, Ls=10, delta=10; assignment to the
20,000 planted centres in both fast precisions).

Checked exactly against the FP64 oracle: every code, every canonical bucket
id, the SILK seed set, and the labels of a random sample of 4,096 points
(the oracle computes each sampled label exhaustively over all centres)."""
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
    bk = ctx.hash(data, cfg.K, cfg.L, a=geek._dev(wl["a"]), b=geek._dev(wl["b"]), w=wl["w"])
    seeds = ctx.silk(bk, **geek.silk_args(wl["silk"]))
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
    assert np.array_equal(g_codes, codes)
    del g_codes
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
