"""The allocation-free dense assignment entry point, called through the C ABI.

Some callers cannot allocate device memory while they run: their memory is
reserved up front by another allocator (a caching pool that already holds
every free byte, so cudaMalloc would fail), or they cannot accept the
implicit synchronisation an allocation or free may cause.
geek_assign_centers_noalloc serves them with a fixed scratch array.  This
test checks its labels, on two calls in a row with different inputs (so the
shared scratch is reused and must be cleared where it has to start at
zero), against the labels of geek_assign_centers in FP32 and against the
oracle's exhaustive FP64 nearest centre, exactly, as every label test here
requires.  It also covers the largest supported d (the largest
shared-memory launch), an odd d, a row stride larger than d and k = 1.  It
is collected last so that a failure here stops a run only after every other
test has run."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(seed, n, d, k, dup):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-10, 10, size=(k, d))
    if dup and k > 1:
        c[k // 2:] = c[: k - k // 2]          # exact ties: smaller index wins
        c[: k // 4] += 1e-9                  # near ties: decided in FP64
    lab = rng.integers(0, k, size=n)
    x = (c[lab] + rng.standard_normal((n, d))).astype(np.float32)
    return x, c


# (seed, n, d, k, exact and near ties, row stride beyond d)
CASES = [
    [(1, 20_011, 32, 300, True, 0), (2, 9_000, 128, 2_000, False, 0)],
    [(3, 3_001, 256, 64, True, 0), (4, 2_000, 37, 50, True, 3)],
    [(5, 1_000, 16, 1, False, 0), (6, 777, 37, 700, True, 5)],
]


@pytest.mark.parametrize("pair", CASES, ids=["d32_d128", "d256_odd_strided", "k1_odd_strided"])
def test_noalloc_matches_assign_centers_and_oracle_twice(pair):
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2106_10515_gb300 import geek
    L = geek.lib()
    ctx = geek.Context(0)
    stream = geek._stream()
    for seed, n, d, k, dup, pad in pair:
        x, c = _case(seed, n, d, k, dup)
        ldx = d + pad
        xfull = np.zeros((n, ldx), dtype=np.float32)
        xfull[:, :d] = x
        xd_full = geek._dev(xfull)
        xd = xd_full[:, :d]                  # row stride ldx on the device
        cd = geek._dev(c)
        want = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assign_centers(ctx.dense(xd), cd, want, precision=geek.PREC_FP32)
        got = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        st = L.geek_assign_centers_noalloc(C.c_void_p(xd_full.data_ptr()), n, d, ldx,
                                           C.c_void_p(cd.data_ptr()), k, C.c_void_p(got.data_ptr()), stream)
        assert st == geek.OK
        torch.cuda.synchronize()
        got_h = got.cpu().numpy()
        assert np.array_equal(got_h, want.cpu().numpy())
        ref, _ = oracle.assign_dense(x, c)
        assert np.array_equal(got_h, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    L = geek.lib()
    x = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    lab = torch.zeros(4, dtype=torch.int32, device="cuda")
    k = 65536 + 1
    c = torch.zeros((k, 16), dtype=torch.float64, device="cuda")
    st = L.geek_assign_centers_noalloc(C.c_void_p(x.data_ptr()), 4, 16, 16, C.c_void_p(c.data_ptr()), k,
                                       C.c_void_p(lab.data_ptr()), geek._stream())
    assert st == geek.ERR_UNSUPPORTED
    c2 = torch.zeros((8, 257), dtype=torch.float64, device="cuda")
    x2 = torch.zeros((4, 257), dtype=torch.float32, device="cuda")
    st = L.geek_assign_centers_noalloc(C.c_void_p(x2.data_ptr()), 4, 257, 257, C.c_void_p(c2.data_ptr()), 8,
                                       C.c_void_p(lab.data_ptr()), geek._stream())
    assert st == geek.ERR_UNSUPPORTED
