"""The tcgen05 dense projection (three-term split BF16, six products per
k-step) against the oracle: E2LSH codes and SRP bits, the canonical buckets
built from them, for every d the kernel takes (a partial k-block, one, two),
row strides beyond d, ragged row tiles, and inputs built to sit on or next to
cell edges with large cancellation.  Every code is exact.  Shapes the kernel
does not take fall back to the FP32 path and stay exact."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
TC = None


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    global TC
    TC = geek.PREC_BF16X3
    return geek


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


def hash_tc(G, ctx, x, a, b, w, K, L, proj=0, pad=0):
    n, d = x.shape
    if pad:
        xf = np.zeros((n, d + pad), dtype=np.float32)
        xf[:, :d] = x
        xd = G._dev(xf)[:, :d]
    else:
        xd = G._dev(x)
    bk = ctx.hash(ctx.dense(xd), K, L, a=G._dev(a), b=G._dev(b), w=w, proj=proj, precision=G.PREC_BF16X3)
    torch.cuda.synchronize()
    return bk


def check(bk, codes_ref, ref):
    got = bk.copy_out()
    assert np.array_equal(got["codes"].cpu().numpy(), codes_ref.astype(np.int32))
    assert np.array_equal(got["obj_bucket"].cpu().numpy(), ref.obj_bucket)
    assert np.array_equal(got["bucket_off"].cpu().numpy(), ref.boff)
    assert np.array_equal(got["members"].cpu().numpy(), ref.bmem)


@pytest.mark.parametrize("n", [1, 4097, 20_000])
def test_tc_projection_small_dense(G, ctx, n):
    wl = synth.make(synth.config("c1", n=n))
    cfg = wl["cfg"]
    bk = hash_tc(G, ctx, wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    codes, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    check(bk, codes, ref)


@pytest.mark.parametrize("w", [2.7, 0.5])
def test_projection_bucket_widths(G, ctx, w):
    """Bucket widths other than the configs' 4: w = 0.5 (a power of two, the
    rechecks divide by an exact multiplication) and w = 2.7 (a true FP64
    division), on both projection forms; many elements land near cell edges."""
    wl = synth.make(synth.config("c1", n=9000))
    cfg = wl["cfg"]
    b = (wl["b"] / 4.0 * w).astype(np.float32)
    codes, ref = oracle.hash_dense(wl["x"], wl["a"], b, w, cfg.K, cfg.L)
    check(hash_tc(G, ctx, wl["x"], wl["a"], b, w, cfg.K, cfg.L), codes, ref)
    bk32 = ctx.hash(ctx.dense(G._dev(wl["x"])), cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(b), w=w)
    torch.cuda.synchronize()
    check(bk32, codes, ref)
    assert bk32.n_flagged > 0


def test_tc_projection_c2_shape(G, ctx):
    """d = 128, 96 functions (K = 6, L = 16), 60,001 rows: several row
    tiles per CTA, a ragged last tile, and elements the window flags."""
    wl = synth.make(synth.config("c2", n=60_001, n_comp=600))
    cfg = wl["cfg"]
    bk = hash_tc(G, ctx, wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    codes, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L)
    check(bk, codes, ref)
    assert bk.n_flagged > 0
    # the window is about as narrow as the FP32 path's
    bk32 = ctx.hash(ctx.dense(G._dev(wl["x"])), cfg.K, cfg.L, a=G._dev(wl["a"]), b=G._dev(wl["b"]), w=wl["w"])
    assert bk.n_flagged <= 2 * bk32.n_flagged + 100


def test_tc_projection_srp(G, ctx):
    wl = synth.make(synth.config("c1", n=9000))
    cfg = wl["cfg"]
    bk = hash_tc(G, ctx, wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L, proj=G.PROJ_SRP)
    bits, ref = oracle.hash_dense(wl["x"], wl["a"], wl["b"], wl["w"], cfg.K, cfg.L, proj="srp")
    check(bk, bits, ref)


@pytest.mark.parametrize("d,K,L,pad", [(20, 4, 8, 0), (64, 4, 8, 4), (96, 5, 6, 0), (100, 3, 10, 8),
                                       (128, 4, 8, 4), (7, 4, 8, 0), (130, 4, 8, 0)])
def test_tc_projection_shapes(G, ctx, d, K, L, pad):
    """Partial and whole k-blocks, F not a multiple of 32 (30 functions),
    strided rows; d = 7 (rows not 16-byte aligned) and d = 130 (> 128)
    take the FP32 path."""
    rng = np.random.default_rng(d * 7 + K)
    n = 5003
    x = (rng.standard_normal((n, d)) * 6).astype(np.float32)
    a = rng.standard_normal((K * L, d)).astype(np.float32)
    b = (rng.random(K * L) * 4).astype(np.float32)
    bk = hash_tc(G, ctx, x, a, b, 4.0, K, L, pad=pad)
    codes, ref = oracle.hash_dense(x, a, b, 4.0, K, L)
    check(bk, codes, ref)


def test_tc_projection_cell_edges_and_cancellation(G, ctx):
    """Rows placed within 1e-4 of a cell edge of one function, and rows
    nearly orthogonal to a function with |x| ~ 1e3 (a.x ~ 0 after large
    cancellation): the fast window must flag them and the recheck decide
    them exactly."""
    rng = np.random.default_rng(77)
    n, d, K, L, w = 8000, 128, 4, 8, 4.0
    F = K * L
    a = rng.standard_normal((F, d)).astype(np.float32)
    b = (rng.random(F) * 4).astype(np.float32)
    x = rng.standard_normal((n, d)) * 30.0
    f = rng.integers(0, F, n)
    af = a[f].astype(np.float64)
    an2 = (af * af).sum(1)
    s = (af * x).sum(1)
    # first half: a_f.x + b_f = m w + eps with |eps| <= 1e-4
    m = np.floor((s + b[f]) / w)
    eps = rng.uniform(-1e-4, 1e-4, n)
    tgt = m * w - b[f] + eps
    h = n // 2
    x[:h] += ((tgt - s) / an2)[:h, None] * af[:h]
    # second half: a_f.x = eps (SRP-style zero crossing) with large |x|
    x[h:] *= 30.0
    s2 = (af[h:] * x[h:]).sum(1)
    x[h:] += ((eps[h:] - s2) / an2[h:])[:, None] * af[h:]
    x = x.astype(np.float32)
    for proj, name in ((G.PROJ_E2LSH, "e2lsh"), (G.PROJ_SRP, "srp")):
        bk = hash_tc(G, ctx, x, a, b, w, K, L, proj=proj)
        codes, ref = oracle.hash_dense(x, a, b, w, K, L, proj=name)
        check(bk, codes, ref)
        assert bk.n_flagged >= n // 4, name


def _tc_coef(d):
    """The kernel's window coefficient (three-term split, per-instruction
    accumulation model), E = coef |a| |x|, plus the 5.02e-7 |a| |x| by which
    the epilogue's one-FFMA cell test widens it to cover its own FP32
    evaluation."""
    nk = (d + 15) // 16
    u20 = 2.0 ** -20
    c = nk * u20 * 1.0079 + 5 * nk * u20 * 0.0079 + 2.0 ** -24 * 1.01 + 2.0 ** -22 * 1.01 + d * 1.12e-16
    return 1.01 * c + 5.02e-7


def test_tc_projection_just_outside_the_window(G, ctx):
    """Elements placed 1.05-1.6 windows from a cell edge, on both sides, with
    |x| ~ 3e3: the kernel settles them without a recheck, so a tensor-core
    accumulation error beyond the modelled bound would show as a wrong code."""
    rng = np.random.default_rng(99)
    n, d, K, L, w = 6000, 128, 4, 8, 4.0
    F = K * L
    a = rng.standard_normal((F, d)).astype(np.float32)
    b = (rng.random(F) * 4).astype(np.float32)
    x = rng.standard_normal((n, d)) * 250.0
    f = rng.integers(0, F, n)
    af = a[f].astype(np.float64)
    an = np.sqrt((af * af).sum(1))
    xn = np.sqrt((x * x).sum(1))
    Et = _tc_coef(d) * an * xn / w                       # the window in cell units
    s = (af * x).sum(1)
    m = np.floor((s + b[f]) / w)
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    frac = np.where(side > 0, 0.0, 1.0) + side * rng.uniform(1.05, 1.6, n) * Et
    tgt = (m + frac) * w - b[f]
    x += ((tgt - s) / (an * an))[:, None] * af
    x = x.astype(np.float32)
    bk = hash_tc(G, ctx, x, a, b, w, K, L)
    codes, ref = oracle.hash_dense(x, a, b, w, K, L)
    check(bk, codes, ref)
    # most of the placed elements stay outside the window after rounding
    # the rows to FP32: they were decided by the tensor-core pass alone
    xs = x.astype(np.float64)
    t_exact = ((af * xs).sum(1) + b[f]) / w
    margin = np.minimum(t_exact - np.floor(t_exact), np.ceil(t_exact) - t_exact) / Et
    assert np.mean((margin > 1.0) & (margin < 2.0)) > 0.5
