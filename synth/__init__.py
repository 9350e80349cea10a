"""Seeded synthetic workloads for the GEEK hash / SILK seed / assign path.

This module only draws random numbers: it holds none of the method's
arithmetic (no hashing, no bucketing, no voting, no distances).  Both the FP64
oracle and the GPU library consume its outputs, so the random parameters that
the method draws (E2LSH projections ``a`` and offsets ``b``, MinHash and SILK
hash coefficients) are produced here and passed to both sides as inputs.

Workload shapes follow the paper's datasets (Sect. 4.1, Table 2): Sift10M-like
dense points (n=10M, d=128), GeoNames-like heterogeneous rows and URL-like
sparse sets.  None of those datasets is available, so every array is drawn
from the recipes below with NumPy's PCG64, one root seed per configuration.

Draw order inside the data stream: mixture centres, then per-component
spreads / weights, then labels, then points (then sets / categorical values).
Hash parameters and SILK coefficients come from separate child streams so
that scaling ``n`` down for a parity case keeps the same parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

ROOT_SEED = 2106105150

# SILK thresholds (K_s, L_s, delta) per workload.  The paper's defaults are
# K=3, delta=10 and L in {10..40} (Sect. 4.2); E2LSH with a fixed width makes
# most buckets singletons on these shapes, so delta is lowered where the
# paper's default would select no seed at all.
SILK_DEFAULTS = {
    "c1": dict(Ks=3, Ls=20, delta=2),
    "c2": dict(Ks=3, Ls=10, delta=10),
    "c3": dict(Ks=3, Ls=20, delta=10),
    "c4": dict(Ks=3, Ls=20, delta=2),
    "c5": dict(Ks=3, Ls=20, delta=2),
}


@dataclass(frozen=True)
class Config:
    name: str
    kind: str                 # "dense" | "sets" | "hetero"
    n: int
    d: int = 0
    n_comp: int = 0
    centre_range: float = 10.0
    sigma: tuple = (1.0, 1.0)  # U[lo, hi] per component and dimension
    weights: str = "equal"     # "equal" | "zipf1"
    K: int = 4
    L: int = 8
    w: float = 4.0
    # sets
    universe: int = 1 << 20
    zipf_items: float = 1.1
    n_base: int = 5000
    set_mean: float = 64.0
    share: float = 0.7
    # hetero
    n_cat: int = 10
    card_range: tuple = (10, 1000)
    zipf_cat: float = 1.2
    Kc: int = 2
    silk: dict = field(default_factory=dict)
    seed: int = ROOT_SEED

    @property
    def F(self) -> int:
        """Number of projection / MinHash functions over all tables."""
        return self.K * self.L


def config(name: str, **over) -> Config:
    """Return workload ``name`` (c1..c4), optionally with fields overridden
    (``n``, ``n_comp`` ... for a smaller parity case of the same shape)."""
    idx = int(name[1:])
    base = {
        "c1": Config("c1", "dense", n=20_000, d=32, n_comp=50, centre_range=10.0,
                     sigma=(1.0, 1.0), weights="equal", K=4, L=8, w=4.0),
        "c2": Config("c2", "dense", n=10_000_000, d=128, n_comp=20_000,
                     centre_range=50.0, sigma=(0.5, 2.0), weights="zipf1",
                     K=6, L=16, w=4.0),
        "c3": Config("c3", "sets", n=2_000_000, K=4, L=32),
        "c4": Config("c4", "hetero", n=2_000_000, d=20, n_comp=2000,
                     centre_range=10.0, sigma=(1.0, 1.0), weights="equal",
                     K=4, L=8, w=4.0, Kc=2),
    }[name]
    cfg = replace(base, silk=dict(SILK_DEFAULTS[name]), seed=ROOT_SEED + idx)
    if over:
        silk_over = over.pop("silk", None)
        cfg = replace(cfg, **over)
        if silk_over:
            cfg = replace(cfg, silk={**cfg.silk, **silk_over})
    return cfg


def _streams(seed: int, key: tuple = ()):
    ss = np.random.SeedSequence(seed, spawn_key=key)
    data, hashp, silk = ss.spawn(3)
    mk = lambda s: np.random.Generator(np.random.PCG64(s))
    return mk(data), mk(hashp), mk(silk)


def _u64(rng, size):
    return rng.integers(0, np.iinfo(np.uint64).max, size=size, dtype=np.uint64,
                        endpoint=True)


def _zipf_cdf(a: float, m: int) -> np.ndarray:
    p = np.arange(1, m + 1, dtype=np.float64) ** (-a)
    c = np.cumsum(p)
    return c / c[-1]


def _zipf_draw(rng, cdf: np.ndarray, size) -> np.ndarray:
    """Ranks 1..len(cdf) with P(r) proportional to r^-a (inverse CDF)."""
    u = rng.random(size)
    return np.searchsorted(cdf, u, side="right").clip(0, len(cdf) - 1) + 1


def dense_points(cfg: Config, rng, chunk: int = 1 << 20):
    """Gaussian mixture: centres U[-R,R]^d, per-component per-dimension sigma
    U[lo,hi], weights equal or proportional to 1/rank (Zipf 1.0 over a random
    rank permutation).  Returns (x float32 [n,d], labels int32, centres f32)."""
    R, d, C = cfg.centre_range, cfg.d, cfg.n_comp
    centres = rng.uniform(-R, R, size=(C, d)).astype(np.float32)
    lo, hi = cfg.sigma
    if lo == hi:
        sig = None
    else:
        sig = rng.uniform(lo, hi, size=(C, d)).astype(np.float32)
    if cfg.weights == "equal":
        labels = rng.integers(0, C, size=cfg.n).astype(np.int32)
    else:
        rank = rng.permutation(C) + 1
        p = 1.0 / rank
        p /= p.sum()
        labels = rng.choice(C, size=cfg.n, p=p).astype(np.int32)
    x = np.empty((cfg.n, d), dtype=np.float32)
    for s in range(0, cfg.n, chunk):
        e = min(cfg.n, s + chunk)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        lab = labels[s:e]
        if sig is None:
            z *= np.float32(lo)
        else:
            z *= sig[lab]
        z += centres[lab]
        x[s:e] = z
    return x, labels, centres


def projection_params(cfg: Config, rng, d: int | None = None):
    """E2LSH functions (Datar et al., named in Sect. 3.1 Remarks):
    a ~ N(0,1)^d and b ~ U[0,w), one per (table, function), float32."""
    d = cfg.d if d is None else d
    a = rng.standard_normal((cfg.F, d), dtype=np.float32)
    b = (rng.random(cfg.F, dtype=np.float32) * np.float32(cfg.w)).astype(np.float32)
    b = np.minimum(b, np.nextafter(np.float32(cfg.w), np.float32(0)))
    return a, b


def minhash_params(rng, count: int):
    """Coefficients (A, B) of count multiply-add-shift hashes, uniform u64."""
    return _u64(rng, count), _u64(rng, count)


def silk_params(cfg: Config, rng):
    s = cfg.silk
    A, B = minhash_params(rng, s["Ls"] * s["Ks"])
    dA, dB = minhash_params(rng, s["Ks"])
    return dict(Ks=s["Ks"], Ls=s["Ls"], delta=s["delta"], mh_a=A, mh_b=B,
                dd_a=dA, dd_b=dB)


def silk_params_slow(sp: dict, mode: str, seed: int = ROOT_SEED + 61) -> dict:
    """A copy of SILK parameters with some multipliers A replaced by values
    in [2^31, 2^31 + 2^20): such a hash climbs by about one half per id, so
    neighbouring ids share its values.  mode "all": every function of the
    even-numbered tables; "first": the first function of every table."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    A = np.array(sp["mh_a"], dtype=np.uint64).copy()
    Ks, Ls = sp["Ks"], sp["Ls"]
    for t in range(Ls):
        for k in range(Ks):
            if (mode == "all" and t % 2 == 0) or (mode == "first" and k == 0):
                A[t * Ks + k] = np.uint64((1 << 31) + int(rng.integers(0, 1 << 20)))
    return dict(sp, mh_a=A)


# The paper's own dense pipeline on the 10M x 128 points: Alg. 1 with m = 40
# QALSH tables of t = 5,000 even buckets (both in the paper's grid), then
# SILK with Ls = 20 (grid) and delta = 10 (default) but Ks = 2: on these
# well-separated mixture components the default Ks = 3 keeps 19 seeds, Ks = 2
# about 1,800 (measured with the oracle).
ALG1 = dict(m=40, t=5_000, Ks=2, Ls=20, delta=10)


def alg1_silk_params(seed: int = ROOT_SEED + 21):
    """SILK coefficients for the Alg. 1 pipeline on the dense points (their
    own stream, so the points and the E2LSH functions stay as drawn)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    A, B = minhash_params(rng, ALG1["Ls"] * ALG1["Ks"])
    dA, dB = minhash_params(rng, ALG1["Ks"])
    return dict(Ks=ALG1["Ks"], Ls=ALG1["Ls"], delta=ALG1["delta"], mh_a=A, mh_b=B, dd_a=dA, dd_b=dB)


def sparse_sets(cfg: Config, rng):
    """URL-like sparse sets (Sect. 4.1): n sets over a universe of 2^20 items,
    items Zipf(1.1) over ranks (item = rank-1); n_base base sets of
    Poisson(64) (min 1) distinct Zipf items; each member picks a cluster
    uniformly, a size s ~ Poisson(64) (min 1), round(0.7 s) items drawn
    without replacement from its base set (capped at the base size) and the
    rest as Zipf items; duplicates are dropped and items sorted.
    Returns (off int64 [n+1], items uint32, labels int32)."""
    cdf = _zipf_cdf(cfg.zipf_items, cfg.universe)
    # base sets: keep drawing until each has its target of distinct items
    bsz = np.maximum(rng.poisson(cfg.set_mean, size=cfg.n_base), 1)
    base = []
    for t in bsz:
        got = np.zeros(0, dtype=np.int64)
        while got.size < t:
            got = np.union1d(got, _zipf_draw(rng, cdf, 2 * int(t)) - 1)
            if got.size > t:
                got = rng.permutation(got)[:t]
                got.sort()
        base.append(got)
    boff = np.zeros(cfg.n_base + 1, dtype=np.int64)
    boff[1:] = np.cumsum([b.size for b in base])
    bitems = np.concatenate(base)
    lab = rng.integers(0, cfg.n_base, size=cfg.n).astype(np.int32)
    s = np.maximum(rng.poisson(cfg.set_mean, size=cfg.n), 1)
    blen = boff[lab + 1] - boff[lab]
    m = np.minimum(np.rint(cfg.share * s).astype(np.int64), blen)
    # m items of the base set without replacement: random keys per base item,
    # keep the m smallest within each member's segment
    seg = np.repeat(np.arange(cfg.n, dtype=np.int64), blen)
    pos = np.arange(seg.size, dtype=np.int64) - np.repeat(np.cumsum(blen) - blen, blen)
    keys = (seg.astype(np.uint64) << np.uint64(32)) | rng.integers(0, 1 << 32, seg.size, dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    rank = np.empty_like(order)
    rank[order] = pos  # rank of each base item within its segment
    keep = rank < np.repeat(m, blen)
    from_base = bitems[np.repeat(boff[lab], blen) + pos][keep]
    seg_base = seg[keep]
    nz = s - m
    seg_z = np.repeat(np.arange(cfg.n, dtype=np.int64), nz)
    from_z = _zipf_draw(rng, cdf, int(nz.sum())) - 1
    allseg = np.concatenate([seg_base, seg_z])
    allit = np.concatenate([from_base, from_z]).astype(np.int64)
    key = np.sort((allseg << 20) | allit)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    sid = key >> 20
    items = (key & ((1 << 20) - 1)).astype(np.uint32)
    off = np.zeros(cfg.n + 1, dtype=np.int64)
    np.add.at(off, sid + 1, 1)
    off = np.cumsum(off)
    return off, items, lab


def categorical(cfg: Config, rng, labels):
    """GeoNames-like categorical attributes (Sect. 4.1): n_cat attributes,
    cardinality floor(exp(U[ln 10, ln 1000])); component c has a home value
    v_cj; a row takes (v_cj + r - 1) mod card_j with r ~ Zipf(1.2) on
    [1, card_j].  Returns (values uint32 [n, n_cat], card int64 [n_cat])."""
    lo, hi = cfg.card_range
    card = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), cfg.n_cat))).astype(np.int64)
    home = np.stack([rng.integers(0, c, size=cfg.n_comp) for c in card], axis=1)
    vals = np.empty((cfg.n, cfg.n_cat), dtype=np.uint32)
    for j, c in enumerate(card):
        r = _zipf_draw(rng, _zipf_cdf(cfg.zipf_cat, int(c)), cfg.n)
        vals[:, j] = ((home[labels, j] + r - 1) % c).astype(np.uint32)
    return vals, card


def make(cfg: Config):
    """Draw one workload.  Returns a dict of NumPy arrays and scalars."""
    rdata, rhash, rsilk = _streams(cfg.seed)
    out = dict(cfg=cfg)
    if cfg.kind in ("dense", "hetero"):
        x, lab, centres = dense_points(cfg, rdata)
        out.update(x=x, labels=lab, centres=centres)
        a, b = projection_params(cfg, rhash)
        out.update(a=a, b=b, w=float(cfg.w))
    if cfg.kind == "hetero":
        vals, card = categorical(cfg, rdata, out["labels"])
        tok_off = np.concatenate([[0], np.cumsum(card)[:-1]]).astype(np.uint32)
        out.update(cat=vals, card=card, tokens=(vals + tok_off[None, :]).astype(np.uint32))
        A, B = minhash_params(rhash, cfg.L * cfg.Kc)
        out.update(mh_a=A, mh_b=B)
    if cfg.kind == "sets":
        off, items, lab = sparse_sets(cfg, rdata)
        out.update(set_off=off, set_items=items, labels=lab)
        A, B = minhash_params(rhash, cfg.F)
        out.update(mh_a=A, mh_b=B)
    out["silk"] = silk_params(cfg, rsilk)
    return out


# ---------------------------------------------------------------------------
# Batched workload: many uneven dense instances (one persistent launch).
# ---------------------------------------------------------------------------
def batch_instances(count: int = 256, n_range=(10_000, 500_000), d_choices=(32, 64, 128),
                    comp_range=(10, 2000), seed: int = ROOT_SEED + 5, n_scale: float = 1.0,
                    threads: int = 1, only=None):
    """``count`` dense instances, n = floor(exp(U[ln 1e4, ln 5e5])) (times
    ``n_scale`` for parity cases), d uniform over {32, 64, 128}, components
    U{10..2000}, centres U[-10,10]^d, sigma = 1, equal weights, E2LSH K=4,
    L=8, w=4 and SILK thresholds as for the small dense workload.  Every
    instance draws from its own stream, so ``threads`` (parallel generation)
    does not change the values, and ``only`` (a list of instance indices)
    returns just those instances, with the same values."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    lo, hi = n_range
    ns = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    ns = np.maximum((ns * n_scale).astype(np.int64), 1)
    ds = rng.choice(np.array(d_choices), size=count)
    cs = rng.integers(comp_range[0], comp_range[1] + 1, size=count)

    def one(i):
        cfg = Config("c5", "dense", n=int(ns[i]), d=int(ds[i]), n_comp=int(cs[i]),
                     centre_range=10.0, sigma=(1.0, 1.0), weights="equal",
                     K=4, L=8, w=4.0, silk=dict(SILK_DEFAULTS["c5"]), seed=seed)
        rdata, rhash, rsilk = _streams(seed, (i,))
        x, lab, centres = dense_points(cfg, rdata)
        a, b = projection_params(cfg, rhash)
        return dict(cfg=cfg, x=x, labels=lab, centres=centres, a=a, b=b,
                    w=float(cfg.w), silk=silk_params(cfg, rsilk))

    idx = list(range(count)) if only is None else [int(i) for i in only]
    if threads <= 1:
        return [one(i) for i in idx]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, idx))
