"""CPU checks of the two facts the SILK grouping's claim path rests on.

MinHash function (Eq. 2's permutation): h(x) = floor(((A x + B) mod 2^64) /
2^32) on the ids x in [0, n) of one instance.

1. Injectivity test: h can repeat a value on [0, n) only if some q in
   [1, n) has A q mod 2^64 within 2^32 of a multiple of 2^64.  So when no q
   has that property, h is one-to-one on [0, n).  Checked against brute force.
2. Matching rule: with function k* one-to-one on the ids, a set B of two or
   more ids shares its Ks-value signature with the one-id set {a} exactly
   when a is B's argmin under k*, a attains B's minimum under every other
   function too, and {a} is one of the one-id sets.  Checked against a search
   over all one-id sets, with functions built to repeat values (multipliers
   near 2^31) mixed in.
"""
import numpy as np

M64 = (1 << 64) - 1


def h(A, B, x):
    return (((A * x + B) & M64) >> 32)


def may_repeat(A, n):
    """Some q in [1, n) with A q mod 2^64 within 2^32 of a multiple of 2^64."""
    for q in range(1, n):
        r = (A * q) & M64
        if r < (1 << 32) or r > (1 << 64) - (1 << 32):
            return True
    return False


def _multipliers(rng, count):
    out = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            out.append(int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2)))  # uniform 64-bit
        elif kind == 1:
            out.append((1 << 31) + int(rng.integers(0, 1 << 20)))  # climbs ~1/2 per id: repeats
        elif kind == 2:
            out.append(int(rng.integers(1, 1 << 33)))  # small: long runs of one value
        else:
            q = int(rng.integers(1, 200))  # A q close to 2^64: repeats at distance q
            out.append(((1 << 64) // q + int(rng.integers(-1000, 1000))) & M64)
    return out


def test_injectivity_criterion_is_sufficient():
    rng = np.random.default_rng(7)
    flagged = 0
    for A in _multipliers(rng, 160):
        n = int(rng.integers(2, 1500))
        B = int(rng.integers(0, 1 << 63)) * 2
        values = [h(A, B, x) for x in range(n)]
        injective = len(set(values)) == n
        if not may_repeat(A, n):
            assert injective, (A, B, n)
        else:
            flagged += 1
        if not injective:
            assert may_repeat(A, n), (A, B, n)  # the contrapositive, stated for clarity
    assert flagged > 40  # the repeating multipliers were caught


def test_one_object_match_rule():
    rng = np.random.default_rng(11)
    Ks = 3
    checked = matched = 0
    for trial in range(40):
        n = int(rng.integers(20, 400))
        coefs = []
        while True:
            As = _multipliers(rng, Ks)
            rng.shuffle(As)
            inj = [k for k in range(Ks) if not may_repeat(As[k], n)]
            if inj:
                break
        Bs = [int(rng.integers(0, 1 << 63)) * 2 for _ in range(Ks)]
        ks = inj[0]
        sig = lambda ids: tuple(min(h(As[k], Bs[k], x) for x in ids) for k in range(Ks))
        ones = set(int(v) for v in rng.choice(n, size=int(rng.integers(1, n)), replace=False))
        one_sig = {}
        for a in ones:
            one_sig.setdefault(sig([a]), []).append(a)
        assert all(len(v) == 1 for v in one_sig.values())  # one-to-one k*: no two share
        for _ in range(60):
            size = int(rng.integers(2, 8))
            bset = [int(v) for v in rng.choice(n, size=size, replace=False)]
            s = sig(bset)
            actual = one_sig.get(s, [None])[0]
            a = min(bset, key=lambda x: h(As[ks], Bs[ks], x))
            rule = a if (all(h(As[k], Bs[k], a) == s[k] for k in range(Ks)) and a in ones) else None
            assert rule == actual, (trial, bset, a, actual)
            checked += 1
            matched += actual is not None
    assert checked == 2400 and matched > 100
