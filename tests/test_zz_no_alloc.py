"""The allocation-free dense assignment entry point, called through the C ABI.

Some callers cannot allocate device memory while they run (their memory is
reserved up front by another allocator, or an allocation's implicit
synchronisation is not acceptable); geek_assign_centers_noalloc serves them
with a fixed scratch array.  This test checks, on two calls in a row with
different inputs (so the shared scratch is reused), that its labels equal
those of geek_assign_centers in FP32, exactly, as every label test here
requires.  It is collected last so that a failure here stops a run only
after every other test has run."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(seed, n, d, k, dup):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-10, 10, size=(k, d))
    if dup:
        c[k // 2:] = c[: k - k // 2]          # exact ties: smaller index wins
        c[: k // 4] += 1e-9                  # near ties: decided in FP64
    lab = rng.integers(0, k, size=n)
    x = (c[lab] + rng.standard_normal((n, d))).astype(np.float32)
    return x, c


def test_noalloc_matches_assign_centers_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_10515_gb300 import geek
    L = geek.lib()
    ctx = geek.Context(0)
    stream = geek._stream()
    for seed, n, d, k, dup in [(1, 20_011, 32, 300, True), (2, 9_000, 128, 2_000, False)]:
        x, c = _case(seed, n, d, k, dup)
        xd, cd = geek._dev(x), geek._dev(c)
        want = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.assign_centers(ctx.dense(xd), cd, want, precision=geek.PREC_FP32)
        got = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        st = L.geek_assign_centers_noalloc(C.c_void_p(xd.data_ptr()), n, d, d, C.c_void_p(cd.data_ptr()), k,
                                           C.c_void_p(got.data_ptr()), stream)
        assert st == geek.OK
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())


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
