"""Python binding of the GEEK C ABI (include/geek.h).

Argument marshalling only: every step runs in libgeek.so's CUDA kernels.
PyTorch provides device memory and the current CUDA stream.  If the library
has not been built, importing this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeek.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_OVERFLOW, ERR_UNSUPPORTED = range(7)
DENSE, SETS, HETERO = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1
PROJ_E2LSH, PROJ_SRP, PROJ_QALSH = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_BF16X3 = 0, 1, 2
PREC_AUTO = -1
OPT_WAIT_LIMIT_NS, OPT_TEST_STALL_TILE, OPT_TEST_FAIL_ALLOC = 1, 2, 3
STATUS_NAMES = ["OK", "ERR_INVALID", "ERR_NOMEM", "ERR_CUDA", "ERR_TIMEOUT", "ERR_OVERFLOW",
                "ERR_UNSUPPORTED"]


class GeekError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class geek_data(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mem", C.c_int32), ("n", C.c_int64), ("d", C.c_int32),
                ("n_cat", C.c_int32), ("ldx", C.c_int64), ("x", C.c_void_p), ("set_off", C.c_void_p),
                ("set_items", C.c_void_p), ("cat", C.c_void_p)]


class geek_hash_params(C.Structure):
    _fields_ = [("proj", C.c_int32), ("precision", C.c_int32), ("K", C.c_int32), ("L", C.c_int32),
                ("Kc", C.c_int32), ("w", C.c_double), ("a", C.c_void_p), ("b", C.c_void_p),
                ("mh_a", C.c_void_p), ("mh_b", C.c_void_p), ("t", C.c_int32), ("doph_bins", C.c_int32),
                ("doph_a", C.c_uint64), ("doph_b", C.c_uint64)]


class geek_buckets_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("L", C.c_int32), ("key_bits_max", C.c_int32),
                ("n_buckets", C.c_int64), ("n_flagged", C.c_int64), ("n_flagged_fp64", C.c_int64)]


class silk_params(C.Structure):
    _fields_ = [("Ks", C.c_int32), ("Ls", C.c_int32), ("delta", C.c_int32), ("mh_a", C.c_void_p),
                ("mh_b", C.c_void_p), ("dd_a", C.c_void_p), ("dd_b", C.c_void_p)]


class geek_assign_params(C.Structure):
    _fields_ = [("precision", C.c_int32)]


class geek_centres_info(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d", C.c_int32), ("n_attr", C.c_int32), ("k", C.c_int64),
                ("n_items", C.c_int64)]


class geek_assign_stats(C.Structure):
    _fields_ = [("sse", C.c_double), ("radius_max", C.c_double), ("k", C.c_int64),
                ("n_recheck_rows", C.c_int64), ("n_fp64_rows", C.c_int64)]


class geek_instance(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("ldx", C.c_int64), ("x", C.c_void_p), ("a", C.c_void_p),
                ("b", C.c_void_p), ("w", C.c_double), ("mh_a", C.c_void_p), ("mh_b", C.c_void_p),
                ("dd_a", C.c_void_p), ("dd_b", C.c_void_p)]


class geek_batch_params(C.Structure):
    _fields_ = [("proj", C.c_int32), ("K", C.c_int32), ("L", C.c_int32), ("Ks", C.c_int32), ("Ls", C.c_int32),
                ("delta", C.c_int32), ("precision", C.c_int32), ("tile_n", C.c_int32)]


class geek_batch_info(C.Structure):
    _fields_ = [("count", C.c_int32), ("n_total", C.c_int64), ("k_total", C.c_int64), ("n_buckets", C.c_int64),
                ("n_flagged", C.c_int64), ("n_flagged_fp64", C.c_int64), ("n_recheck_rows", C.c_int64),
                ("key_bits", C.c_int32), ("graph_launches", C.c_int32), ("graph_captures", C.c_int32),
                ("tuned_classes", C.c_int32), ("n_fp64_rows", C.c_int64)]


# every symbol declared in include/geek.h
EXPORTS = ["geek_ctx_create", "geek_ctx_destroy", "geek_last_error", "geek_version", "geek_hash",
           "geek_buckets_info_get", "geek_buckets_copy_out", "geek_buckets_free", "silk_seed",
           "silk_seeds_info", "silk_seeds_copy_out", "silk_seeds_free", "geek_assign",
           "geek_assign_centers", "geek_timing_enable", "geek_timing_reset", "geek_timing_get",
           "geek_launch_count", "geek_assign_centers_noalloc", "geek_batch_create", "geek_batch_run",
           "geek_batch_info_get", "geek_batch_instance_stats", "geek_batch_copy_out", "geek_batch_seed_ids_count",
           "geek_batch_destroy", "geek_data_upload", "geek_resident_free", "geek_refine",
           "geek_ctx_set_option", "geek_assign_ex", "geek_centres_info_get", "geek_centres_copy_out",
           "geek_centres_free", "geek_cluster_radius"]

_lib = None


def lib():
    """Loads libgeek.so (raises if it was never built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    P, st = C.c_void_p, C.c_int
    L.geek_ctx_create.argtypes = [C.c_int, C.POINTER(P)]
    L.geek_ctx_destroy.argtypes = [P]
    L.geek_last_error.argtypes = [P]
    L.geek_last_error.restype = C.c_char_p
    L.geek_version.restype = C.c_char_p
    L.geek_hash.argtypes = [P, C.POINTER(geek_data), C.POINTER(geek_hash_params), C.POINTER(P), P]
    L.geek_buckets_info_get.argtypes = [P, C.POINTER(geek_buckets_info)]
    L.geek_buckets_copy_out.argtypes = [P, P, P, P, P, P, P]
    L.geek_buckets_free.argtypes = [P]
    L.silk_seed.argtypes = [P, P, C.POINTER(silk_params), C.POINTER(P), P]
    L.silk_seeds_info.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.silk_seeds_copy_out.argtypes = [P, P, P, P]
    L.silk_seeds_free.argtypes = [P]
    L.geek_assign.argtypes = [P, C.POINTER(geek_data), P, P, C.POINTER(geek_assign_params), P, P,
                              C.POINTER(geek_assign_stats), P]
    L.geek_assign_centers.argtypes = [P, C.POINTER(geek_data), P, C.c_int64,
                                      C.POINTER(geek_assign_params), P, C.POINTER(geek_assign_stats), P]
    L.geek_ctx_set_option.argtypes = [P, C.c_int32, C.c_int64]
    L.geek_cluster_radius.argtypes = [P, C.POINTER(geek_data), P, C.c_int64, P, P, P]
    L.geek_assign_ex.argtypes = [P, C.POINTER(geek_data), P, P, C.POINTER(geek_assign_params), P,
                                 C.POINTER(geek_assign_stats), C.POINTER(P), P]
    L.geek_centres_info_get.argtypes = [P, C.POINTER(geek_centres_info)]
    L.geek_centres_copy_out.argtypes = [P, P, P, P, P, P]
    L.geek_centres_free.argtypes = [P]
    L.geek_timing_enable.argtypes = [P, C.c_int]
    L.geek_timing_reset.argtypes = [P]
    L.geek_timing_get.argtypes = [P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double)]
    L.geek_launch_count.restype = C.c_ulonglong
    L.geek_assign_centers_noalloc.argtypes = [P, C.c_int64, C.c_int32, C.c_int64, P, C.c_int64, P, P]
    L.geek_batch_create.argtypes = [P, C.POINTER(geek_instance), C.c_int32, C.POINTER(geek_batch_params),
                                    C.POINTER(P)]
    L.geek_batch_run.argtypes = [P, P, P]
    L.geek_batch_info_get.argtypes = [P, C.POINTER(geek_batch_info)]
    L.geek_batch_instance_stats.argtypes = [P, P, P, P, P, P]
    L.geek_batch_copy_out.argtypes = [P, P, P, P, P, P, P]
    L.geek_batch_seed_ids_count.argtypes = [P, C.POINTER(C.c_int64)]
    L.geek_batch_destroy.argtypes = [P]
    L.geek_data_upload.argtypes = [P, C.POINTER(geek_data), C.POINTER(P), C.POINTER(geek_data), P]
    L.geek_resident_free.argtypes = [P]
    L.geek_refine.argtypes = [P, C.POINTER(geek_data), P, C.c_int64, C.c_int32, C.POINTER(geek_assign_params), P,
                              C.POINTER(geek_assign_stats), P]
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("geek_last_error", "geek_version", "geek_ctx_destroy", "geek_launch_count"):
            f.restype = st
    _lib = L
    return L


def version() -> str:
    return lib().geek_version().decode()


def launch_count() -> int:
    return int(lib().geek_launch_count())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr() if t.numel() else None
    if isinstance(t, np.ndarray):
        return t.ctypes.data if t.size else None
    raise TypeError(type(t))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(a, dtype=None):
    """numpy / tensor -> contiguous CUDA tensor (uint64 arrays as int64 bits)."""
    if isinstance(a, np.ndarray):
        if a.dtype == np.uint64:
            a = a.view(np.int64)
        a = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None and a.dtype != dtype:
        a = a.to(dtype)
    return a.contiguous().cuda()


class Data:
    """A geek_data descriptor plus references that keep its arrays alive."""

    def __init__(self, kind, host, n, refs):
        self.c = geek_data()
        self.c.kind, self.c.mem, self.c.n = kind, MEM_HOST if host else MEM_DEVICE, n
        self.refs = refs

    @classmethod
    def dense(cls, x, host=False):
        self = cls(DENSE, host, x.shape[0], [x])
        self.c.d = x.shape[1]
        # a row-strided view (unit column stride) passes its row stride
        if isinstance(x, torch.Tensor) and x.dim() == 2 and x.stride(1) == 1 and x.shape[0] > 1:
            self.c.ldx = x.stride(0)
        else:
            self.c.ldx = x.shape[1]
        self.c.x = _ptr(x)
        return self

    @classmethod
    def sets(cls, off, items, host=False):
        self = cls(SETS, host, off.shape[0] - 1, [off, items])
        self.c.set_off, self.c.set_items = _ptr(off), _ptr(items)
        return self

    @classmethod
    def hetero(cls, x, tokens, host=False):
        self = cls.dense(x, host)
        self.c.kind = HETERO
        self.c.n_cat = tokens.shape[1]
        self.c.cat = _ptr(tokens)
        self.refs.append(tokens)
        return self


class Resident:
    """Library-owned device copy of a host data set (geek_data_upload); the
    buffers are reused by the next upload into the same handle."""

    def __init__(self, ctx):
        self.ctx, self.h = ctx, C.c_void_p()
        self.data = None

    def upload(self, host: Data) -> Data:
        """Copies `host` (a Data with host=True) in stream order; returns the
        device view, valid until the next upload or the handle's release."""
        v = Data(host.c.kind, False, host.c.n, [self, host])
        self.ctx._chk(lib().geek_data_upload(self.ctx.h, C.byref(host.c), C.byref(self.h), C.byref(v.c),
                                             _stream()))
        self.data = v
        return v

    def __del__(self):
        if self.h:
            lib().geek_resident_free(self.h)
            self.h = C.c_void_p()


class Buckets:
    """geek_hash result (library-owned)."""

    def __init__(self, ctx, handle, F):
        self.ctx, self.h, self.F = ctx, handle, F
        info = geek_buckets_info()
        ctx._chk(lib().geek_buckets_info_get(self.h, C.byref(info)))
        self.n, self.L = info.n, info.L
        self.key_bits_max, self.n_buckets, self.n_flagged = info.key_bits_max, info.n_buckets, info.n_flagged
        self.n_flagged_fp64 = info.n_flagged_fp64

    def copy_out(self):
        n, L = self.n, self.L
        ob = torch.empty((L, n), dtype=torch.int32, device="cuda")
        nb = np.zeros(L, dtype=np.int64)
        boff = torch.empty(self.n_buckets + 1, dtype=torch.int64, device="cuda")
        mem = torch.empty(L * n, dtype=torch.int32, device="cuda")
        codes = torch.empty((n, self.F), dtype=torch.int32, device="cuda")
        self.ctx._chk(lib().geek_buckets_copy_out(self.h, _ptr(ob), nb.ctypes.data, _ptr(boff), _ptr(mem),
                                                  _ptr(codes), _stream()))
        return dict(obj_bucket=ob, n_buckets=nb, bucket_off=boff, members=mem, codes=codes)

    def __del__(self):
        if getattr(self, "h", None):
            lib().geek_buckets_free(self.h)
            self.h = None


class Seeds:
    def __init__(self, ctx, handle):
        self.ctx, self.h = ctx, handle
        k, ni, nm = C.c_int64(), C.c_int64(), C.c_int64()
        ctx._chk(lib().silk_seeds_info(self.h, C.byref(k), C.byref(ni), C.byref(nm)))
        self.k, self.n_ids, self.n_multiset = k.value, ni.value, nm.value

    def copy_out(self):
        off = torch.empty(self.k + 1, dtype=torch.int64, device="cuda")
        ids = torch.empty(max(self.n_ids, 1), dtype=torch.int32, device="cuda")
        self.ctx._chk(lib().silk_seeds_copy_out(self.h, _ptr(off), _ptr(ids), _stream()))
        return off, ids[: self.n_ids]

    def sets(self):
        off, ids = self.copy_out()
        off, ids = off.cpu().numpy(), ids.cpu().numpy()
        return [tuple(ids[off[j]:off[j + 1]].tolist()) for j in range(self.k)]

    def __del__(self):
        if getattr(self, "h", None):
            lib().silk_seeds_free(self.h)
            self.h = None


class Context:
    """One GEEK context on a CUDA device."""

    def __init__(self, device: int = 0):
        torch.cuda.set_device(device)
        h = C.c_void_p()
        st = lib().geek_ctx_create(device, C.byref(h))
        if st != OK:
            raise GeekError(st, f"geek_ctx_create(device={device}) failed")
        self.h = h
        self._keep = []

    def set_option(self, option, value):
        self._chk(lib().geek_ctx_set_option(self.h, option, int(value)))

    def timing(self, on=True):
        self._chk(lib().geek_timing_enable(self.h, 1 if on else 0))

    def timing_reset(self):
        self._chk(lib().geek_timing_reset(self.h))

    def timing_get(self, name):
        """(total ms, brackets, total algorithmic work) recorded under name."""
        ms, cnt, work = C.c_double(), C.c_int64(), C.c_double()
        self._chk(lib().geek_timing_get(self.h, name.encode(), C.byref(ms), C.byref(cnt), C.byref(work)))
        return ms.value, cnt.value, work.value

    def _chk(self, st):
        if st != OK:
            raise GeekError(st, lib().geek_last_error(self.h).decode())

    def __del__(self):
        if getattr(self, "h", None):
            lib().geek_ctx_destroy(self.h)
            self.h = None

    # ---------------------------------------------------------------- data --
    def resident(self) -> "Resident":
        return Resident(self)

    @staticmethod
    def dense(x, host=False):
        return Data.dense(x, host)

    @staticmethod
    def sets(off, items, host=False):
        return Data.sets(off, items, host)

    @staticmethod
    def hetero(x, tokens, host=False):
        return Data.hetero(x, tokens, host)

    # ---------------------------------------------------------------- hash --
    def hash(self, data, K, L, a=None, b=None, w=4.0, mh_a=None, mh_b=None, Kc=0,
             proj=PROJ_E2LSH, precision=PREC_FP32, t=0, doph_bins=0, doph_a=0, doph_b=0) -> Buckets:
        p = geek_hash_params()
        p.proj, p.precision, p.K, p.L, p.Kc, p.w, p.t = proj, precision, K, L, Kc, float(w), t
        p.doph_bins, p.doph_a, p.doph_b = doph_bins, int(doph_a), int(doph_b)
        p.a, p.b, p.mh_a, p.mh_b = _ptr(a), _ptr(b), _ptr(mh_a), _ptr(mh_b)
        out = C.c_void_p()
        self._chk(lib().geek_hash(self.h, C.byref(data.c), C.byref(p), C.byref(out), _stream()))
        F = K * L
        return Buckets(self, out, F)

    def silk(self, buckets: Buckets, Ks, Ls, delta, mh_a, mh_b, dd_a, dd_b) -> Seeds:
        p = silk_params()
        p.Ks, p.Ls, p.delta = Ks, Ls, delta
        p.mh_a, p.mh_b, p.dd_a, p.dd_b = _ptr(mh_a), _ptr(mh_b), _ptr(dd_a), _ptr(dd_b)
        out = C.c_void_p()
        self._chk(lib().silk_seed(self.h, buckets.h, C.byref(p), C.byref(out), _stream()))
        return Seeds(self, out)

    def assign(self, data, buckets, seeds: Seeds, labels, centers=None, precision=PREC_FP32, stats=True):
        p = geek_assign_params()
        p.precision = precision
        s = geek_assign_stats()
        self._chk(lib().geek_assign(self.h, C.byref(data.c), buckets.h if buckets is not None else None,
                                    seeds.h, C.byref(p), _ptr(labels), _ptr(centers),
                                    C.byref(s) if stats else None, _stream()))
        return s

    def assign_ex(self, data, buckets, seeds, labels, precision=PREC_FP32):
        """geek_assign_ex: labels, stats and the central vectors used, as a
        dict of CUDA tensors ("centers" k x d, or "modes" k x n_attr, or
        "item_off" / "items")."""
        p = geek_assign_params()
        p.precision = precision
        s = geek_assign_stats()
        h = C.c_void_p()
        self._chk(lib().geek_assign_ex(self.h, C.byref(data.c), buckets.h if buckets is not None else None,
                                       seeds.h, C.byref(p), _ptr(labels), C.byref(s), C.byref(h), _stream()))
        try:
            info = geek_centres_info()
            self._chk(lib().geek_centres_info_get(h, C.byref(info)))
            out = {"kind": info.kind, "k": info.k}
            cen = mod = off = items = None
            if info.kind == DENSE:
                cen = torch.empty((info.k, info.d), dtype=torch.float64, device="cuda")
                out["centers"] = cen
            elif info.kind == HETERO or info.n_attr > 0:  # modes (heterogeneous rows, DOPH-reduced sets)
                mod = torch.empty((info.k, info.n_attr), dtype=torch.int64, device="cuda")
                out["modes"] = mod
            else:
                off = torch.empty(info.k + 1, dtype=torch.int64, device="cuda")
                items = torch.empty(max(info.n_items, 1), dtype=torch.int32, device="cuda")
                out["item_off"], out["items"] = off, items[: info.n_items]
            self._chk(lib().geek_centres_copy_out(h, _ptr(cen), _ptr(mod), _ptr(off), _ptr(items), _stream()))
            torch.cuda.synchronize()
        finally:
            lib().geek_centres_free(h)
        return s, out

    def refine(self, data, centers, labels, passes, precision=PREC_FP32, stats=True):
        """Sect. 5's extra passes of assignment: centers (k x d float64) and
        labels (n int32) on the device, updated in place."""
        p = geek_assign_params()
        p.precision = precision
        s = geek_assign_stats() if stats else None
        self._chk(lib().geek_refine(self.h, C.byref(data.c), _ptr(centers), centers.shape[0], passes, C.byref(p),
                                    _ptr(labels), C.byref(s) if s is not None else None, _stream()))
        return s

    def assign_centers(self, data, centers, labels, precision=PREC_FP32, stats=True):
        p = geek_assign_params()
        p.precision = precision
        s = geek_assign_stats()
        k = centers.shape[0]
        self._chk(lib().geek_assign_centers(self.h, C.byref(data.c), _ptr(centers), k, C.byref(p), _ptr(labels),
                                            C.byref(s) if stats else None, _stream()))
        return s

    def cluster_radius(self, data, centers, labels, radius):
        """radius[j] = largest distance of an object labelled j to centre j
        (device buffers; radius: k float64)."""
        self._chk(lib().geek_cluster_radius(self.h, C.byref(data.c), _ptr(centers), centers.shape[0], _ptr(labels),
                                            _ptr(radius), _stream()))


def silk_args(sp):
    """Device copies of a SILK parameter dict (from synth.silk_params)."""
    return dict(Ks=sp["Ks"], Ls=sp["Ls"], delta=sp["delta"], mh_a=_dev(sp["mh_a"]), mh_b=_dev(sp["mh_b"]),
                dd_a=_dev(sp["dd_a"]), dd_b=_dev(sp["dd_b"]))


class Batch:
    """A batch of dense instances (geek_batch): one plan, runs replayed.

    ``instances`` is a list of dicts with device tensors x (n x d float32),
    a (K*L x d float32), b (K*L float32), mh_a / mh_b (Ls*Ks int64 bits of
    uint64), dd_a / dd_b (Ks), and w.  The tensors are kept alive here."""

    def __init__(self, ctx: Context, instances, K, L, Ks, Ls, delta, proj=PROJ_E2LSH, tile_n=0, precision=PREC_AUTO):
        self.ctx = ctx
        self._refs = instances
        arr = (geek_instance * len(instances))()
        for c, I in zip(arr, instances):
            x = I["x"]
            c.n, c.d, c.ldx = x.shape[0], x.shape[1], x.shape[1]
            c.x, c.a, c.b, c.w = _ptr(x), _ptr(I["a"]), _ptr(I["b"]), float(I["w"])
            c.mh_a, c.mh_b, c.dd_a, c.dd_b = _ptr(I["mh_a"]), _ptr(I["mh_b"]), _ptr(I["dd_a"]), _ptr(I["dd_b"])
        p = geek_batch_params()
        p.proj, p.K, p.L, p.Ks, p.Ls, p.delta, p.tile_n = proj, K, L, Ks, Ls, delta, tile_n
        p.precision = precision
        h = C.c_void_p()
        ctx._chk(lib().geek_batch_create(ctx.h, arr, len(instances), C.byref(p), C.byref(h)))
        self.h = h
        self.count = len(instances)
        self.K, self.L = K, L
        self.ns = [I["x"].shape[0] for I in instances]
        self.ds = [I["x"].shape[1] for I in instances]
        self.row_off = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)

    def run(self, labels):
        self.ctx._chk(lib().geek_batch_run(self.h, _ptr(labels), _stream()))

    def info(self):
        i = geek_batch_info()
        self.ctx._chk(lib().geek_batch_info_get(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in geek_batch_info._fields_}

    def instance_stats(self):
        n = self.count
        k, sse, rmax = np.zeros(n, np.int64), np.zeros(n, np.float64), np.zeros(n, np.float64)
        tile, prec = np.zeros(n, np.int32), np.zeros(n, np.int32)
        self.ctx._chk(lib().geek_batch_instance_stats(self.h, k.ctypes.data, sse.ctypes.data, rmax.ctypes.data,
                                                      tile.ctypes.data, prec.ctypes.data))
        return dict(k=k, sse=sse, radius_max=rmax, tile_n=tile, precision=prec)

    def copy_out(self):
        """Per-instance results of the last run (host numpy)."""
        st = self.instance_stats()
        N = int(self.row_off[-1])
        kt = int(st["k"].sum())
        nid = C.c_int64()
        self.ctx._chk(lib().geek_batch_seed_ids_count(self.h, C.byref(nid)))
        codes = torch.empty((N, self.K * self.L), dtype=torch.int32, device="cuda")
        ob = torch.empty((self.L, N), dtype=torch.int32, device="cuda")
        soff = torch.empty(kt + 1, dtype=torch.int64, device="cuda")
        sids = torch.empty(max(nid.value, 1), dtype=torch.int32, device="cuda")
        kd = int(sum(int(k) * d for k, d in zip(st["k"], self.ds)))
        cen = torch.empty(max(kd, 1), dtype=torch.float64, device="cuda")
        self.ctx._chk(lib().geek_batch_copy_out(self.h, _ptr(codes), _ptr(ob), _ptr(soff), _ptr(sids), _ptr(cen),
                                                _stream()))
        codes, ob, soff = codes.cpu().numpy(), ob.cpu().numpy(), soff.cpu().numpy()
        sids, cen = sids.cpu().numpy()[: nid.value], cen.cpu().numpy()
        out = []
        sb = np.concatenate([[0], np.cumsum(st["k"])])
        co = np.concatenate([[0], np.cumsum(st["k"] * np.array(self.ds))])
        for i in range(self.count):
            r0, r1 = self.row_off[i], self.row_off[i + 1]
            s0, s1 = sb[i], sb[i + 1]
            seeds = [tuple(sids[soff[j]:soff[j + 1]].tolist()) for j in range(s0, s1)]
            out.append(dict(codes=codes[r0:r1], obj_bucket=ob[:, r0:r1], seeds=seeds,
                            centres=cen[co[i]:co[i + 1]].reshape(int(st["k"][i]), self.ds[i]),
                            k=int(st["k"][i]), sse=float(st["sse"][i]), radius_max=float(st["radius_max"][i]),
                            tile_n=int(st["tile_n"][i])))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib().geek_batch_destroy(self.h)
            self.h = None
