"""Error paths of the library on the GPU, without faulting it.

A bounded device wait that runs out must come back as GEEK_ERR_TIMEOUT and
leave the context usable; a failed device allocation must come back as
GEEK_ERR_NOMEM.  Both failures are injected through context options: a
radix-sort tile that never publishes its count (its successors' waits run
out after a 1 ms limit, so nothing hangs), and a countdown after which an
allocation reports failure on the host.  After each failure the same
context, and a fresh one, still give the oracle's bucket ids."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    return geek


def _wl():
    # several radix tiles per table (a tile holds 2560 keys)
    return synth.make(synth.config("c1", n=20_000))


def _hash(G, ctx, wl):
    cfg = wl["cfg"]
    return ctx.hash(ctx.dense(G._dev(wl["x"])), cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=wl["w"])


def _check_ok(G, ctx, wl, ref):
    bk = _hash(G, ctx, wl)
    torch.cuda.synchronize()
    assert np.array_equal(bk.copy_out()["obj_bucket"].cpu().numpy(), ref.obj_bucket)


def test_lookback_wait_runs_out_and_reports_timeout(G):
    wl = _wl()
    cfg = wl["cfg"]
    ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)[1]
    ctx = G.Context(0)
    ctx.set_option(G.OPT_WAIT_LIMIT_NS, 1_000_000)   # 1 ms
    ctx.set_option(G.OPT_TEST_STALL_TILE, 2)
    with pytest.raises(G.GeekError) as e:
        _hash(G, ctx, wl)
    assert e.value.status == G.ERR_TIMEOUT
    torch.cuda.synchronize()                          # the context is still usable
    ctx.set_option(G.OPT_TEST_STALL_TILE, -1)
    _check_ok(G, ctx, wl, ref)
    _check_ok(G, G.Context(0), wl, ref)


def test_allocation_failure_reports_nomem(G):
    wl = _wl()
    cfg = wl["cfg"]
    ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)[1]
    ctx = G.Context(0)
    for after in (0, 3, 10):
        ctx.set_option(G.OPT_TEST_FAIL_ALLOC, after)
        with pytest.raises(G.GeekError) as e:
            _hash(G, ctx, wl)
        assert e.value.status == G.ERR_NOMEM
        assert "injected" in str(e.value)
    torch.cuda.synchronize()
    _check_ok(G, ctx, wl, ref)


def test_options_are_checked(G):
    ctx = G.Context(0)
    for opt, val in ((G.OPT_WAIT_LIMIT_NS, 10), (G.OPT_TEST_STALL_TILE, -2), (G.OPT_TEST_FAIL_ALLOC, -5), (99, 0)):
        with pytest.raises(G.GeekError) as e:
            ctx.set_option(opt, val)
        assert e.value.status == G.ERR_INVALID
