"""CPU model of the SILK grouping tables' concurrent protocol, run under random
interleavings of its shared-memory steps.

Each set of two or more objects inserts itself into an open-addressing table
of 64-bit slots (32-bit fingerprint | first set of the group, top bit of the
low word = the group holds >= 2 sets): it reads a slot (the first read may be
stale by the time it acts), claims an empty one by compare-and-swap, or, on a
fingerprint match, compares the owner's full signature and joins.  A joiner
appends itself to the bin list; whoever first sets the group bit also
appends the group's first set; a set that shares its signature with a
one-object bucket claims that bucket in a bit map, and the one claimant
appends it (and the first set, if it set the group bit first).  Every step
that touches shared state is one atomic action here, and a scheduler picks
which set moves next at random.

The bin list must hold every group of two or more sets (one-object buckets
included) exactly once per member, and nothing else.
"""
import random
from collections import Counter, defaultdict

EMPTY = (1 << 64) - 1
MULTI = 1 << 31


def _set_thread(g, sig, fp, home, mask, gi, shared, out):
    """Generator: one set's insertion; yields before every shared access."""
    slots, sigs, claimed = shared["slots"], shared["sigs"], shared["claimed"]
    mine = (fp << 32) | g
    h = home
    yield
    cur = slots[h]  # first read, issued early: may be stale below
    key = owner = None
    joined = first = False
    for probe in range(mask + 1):
        if probe:
            yield
            cur = slots[h]
        if cur == EMPTY:
            yield
            prev = slots[h]  # atomicCAS
            if prev == EMPTY:
                slots[h] = mine
                key, owner = h, g
                break
            cur = prev
        if (cur >> 32) == fp:
            r = cur & 0xFFFFFFFF & ~MULTI
            yield
            if sigs[r] == sig:  # owner's signature, written before the table was used
                if not (cur & MULTI):
                    yield
                    old = slots[h]  # atomicOr
                    slots[h] = old | MULTI
                    first = not (old & MULTI)
                key, owner, joined = h, r, True
                break
        h = (h + 1) & mask
    if joined:
        out.append((key, g))
    if first:
        out.append((key, owner))
    if gi is not None:
        yield
        if not claimed.get(gi, False):  # atomicOr on the claim bit
            claimed[gi] = True
            out.append((key, gi))
            yield
            old = slots[key]  # atomicOr on the group bit
            slots[key] = old | MULTI
            if not (old & MULTI):
                out.append((key, owner))


def _run(seed):
    rng = random.Random(seed)
    n_multi = rng.randint(2, 40)
    n_sig = rng.randint(1, max(1, n_multi // 2))
    C = 64
    while C < 2 * n_multi:
        C <<= 1
    mask = C - 1
    # set ids: one-object buckets 0 .. n_one-1, sets of two or more after them
    n_one = rng.randint(0, 10)
    sig_of = [rng.randrange(n_sig) for _ in range(n_multi)]
    # fingerprints: equal for equal signatures, and colliding on purpose
    fp_of_sig = [rng.randrange(3) for _ in range(n_sig)]
    home_of_sig = [rng.randrange(C) for _ in range(n_sig)]
    one_sig = {}  # one-object bucket -> the signature it shares (at most one bucket per signature)
    sigs_with_one = rng.sample(range(n_sig), min(n_one, n_sig))
    for b, s in enumerate(sigs_with_one):
        one_sig[b] = s
    sig_to_one = {s: b for b, s in one_sig.items()}
    shared = {"slots": [EMPTY] * C, "sigs": {}, "claimed": {}}
    for m in range(n_multi):
        shared["sigs"][n_one + m] = sig_of[m]
    out = []
    threads = []
    for m in range(n_multi):
        g = n_one + m
        s = sig_of[m]
        threads.append(_set_thread(g, s, fp_of_sig[s], home_of_sig[s], mask, sig_to_one.get(s), shared, out))
    live = list(threads)
    while live:
        t = rng.choice(live)
        try:
            next(t)
        except StopIteration:
            live.remove(t)
    # expected groups: signature -> its sets of two or more objects and its one-object bucket
    members = defaultdict(list)
    for m in range(n_multi):
        members[sig_of[m]].append(n_one + m)
    for b, s in one_sig.items():
        if s in members:
            members[s].append(b)
    expect = Counter()
    for s, mem in members.items():
        if len(mem) >= 2:
            for g in mem:
                expect[(s, g)] += 1
    got = Counter()
    key_sig = {}
    for key, g in out:
        s = shared["sigs"].get(g, one_sig.get(g))
        assert key_sig.setdefault(key, s) == s, "one slot key holds two signatures"
        got[(s, g)] += 1
    assert got == expect, (seed, got - expect, expect - got)


def test_grouping_protocol_under_random_interleavings():
    for seed in range(3000):
        _run(seed)
