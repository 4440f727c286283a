"""Thin Python binding of the C ABI in ``include/sws.h``.

Argument marshalling only: torch tensors supply device memory (``data_ptr()``) and the current
CUDA stream; every step of the computation runs in the CUDA library.  If the library has not
been built, every call raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

OPS = {"add_i32": 0, "min_i32": 1, "max_i32": 2, "xor_i32": 3, "affine_u32": 4, "add_f32": 5}
VARIANTS = {"auto": 0, "block_combine": 1, "doubling": 2, "prefix_diff": 3, "stream": 4, "warp": 5}
KMER_KINDS = {"fwd": 0, "rc": 1, "canonical": 2, "hash": 3}
MINI_MODES = {"hash": 0, "canonical": 1, "fwd": 2}

SWS_OK = 0
SWS_ERR_CAPACITY = 3
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CAPACITY", 4: "CUDA", 5: "TIMEOUT", 6: "UNSUPPORTED"}

_lock = threading.Lock()
_lib = None
_ctx = {}

vp = ctypes.c_void_p
u64 = ctypes.c_uint64
i32 = ctypes.c_int


class SwsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sws error {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# name -> (restype, argtypes): every entry point of include/sws.h
SIGNATURES = {
    "sws_last_error": (ctypes.c_char_p, []),
    "sws_create": (i32, [ctypes.POINTER(vp), i32]),
    "sws_destroy": (i32, [vp]),
    "sws_reserve": (i32, [vp, u64]),
    "sws_sync": (i32, [vp, vp]),
    "sws_sliding_sum": (i32, [vp, i32, i32, vp, vp, u64, i32, vp]),
    "sws_tune_sliding_sum": (i32, [vp, i32, i32, u64, vp, vp, vp]),
    "sws_selftest_wait_timeout": (i32, [vp, i32, vp]),
    "sws_selftest_minimizer_timeout": (i32, [vp, vp, vp]),
    "sws_minimizer_strands": (i32, [vp, vp, u64, i32, vp, vp, u64, vp, u64, vp, vp]),
    "sws_seed_lookup": (i32, [vp, vp, u64, i32, i32, vp, vp, u64, vp, vp, vp]),
    "sws_seed_hits": (i32, [vp, vp, vp, u64, ctypes.c_uint32, vp, vp, vp, u64, vp, vp]),
    "sws_kmers": (i32, [vp, vp, u64, i32, i32, vp, vp]),
    "sws_minimizers": (i32, [vp, vp, u64, i32, i32, i32, vp, u64, vp, vp, u64, vp, vp]),
    "sws_minimizers_from_keys": (i32, [vp, vp, u64, i32, vp, vp, u64, vp, vp]),
    "sws_minimizers_count": (i32, [vp, vp, u64, i32, i32, i32, vp, u64, vp, vp]),
    "sws_build_table": (i32, [vp, vp, u64, i32, i32, i32, vp, u64, i32, vp, vp, u64, vp, ctypes.POINTER(u64), vp]),
    "sws_minimizers_batch": (i32, [vp, vp, vp, u64, u64, i32, i32, i32, vp, vp, u64, vp, vp, vp]),
    "sws_kmer_table": (i32, [vp, vp, vp, u64, i32, i32, vp, vp, vp, vp]),
    "sws_minimizers_noalloc": (i32, [vp, u64, i32, i32, i32, vp, u64, vp, vp, u64, vp, vp]),
    "sws_batch_create": (i32, [vp, u64, u64, i32, i32, i32, i32, ctypes.POINTER(vp)]),
    "sws_batch_destroy": (i32, [vp]),
    "sws_batch_io_get": (i32, [vp, vp]),
    "sws_batch_run": (i32, [vp, u64, u64, vp]),
    "sws_batch_sync": (i32, [vp]),
    "sws_server_create": (i32, [vp, vp, ctypes.POINTER(vp)]),
    "sws_server_submit": (i32, [vp, vp, u64, ctypes.POINTER(u64)]),
    "sws_server_submit_batch": (i32, [vp, vp, vp, u64, vp]),
    "sws_server_wait": (i32, [vp, u64, ctypes.c_double, ctypes.POINTER(i32)]),
    "sws_server_result": (i32, [vp, u64, vp, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double)]),
    "sws_server_collect": (i32, [vp, u64, ctypes.c_double, vp, vp, vp, vp, vp, ctypes.POINTER(u64)]),
    "sws_server_release": (i32, [vp, vp, u64]),
    "sws_server_stats": (i32, [vp, vp]),
    "sws_server_reset_stats": (i32, [vp]),
    "sws_server_destroy": (i32, [vp]),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("k", i32), ("w", i32), ("mode", i32), ("slots", ctypes.c_uint32), ("max_requests_per_batch", u64),
                ("max_bases_per_batch", u64), ("hbm_budget_bytes", u64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", u64), ("batches", u64), ("bases", u64), ("pending", u64), ("p50_s", ctypes.c_double),
                ("p99_s", ctypes.c_double), ("max_s", ctypes.c_double), ("mean_s", ctypes.c_double),
                ("span_s", ctypes.c_double)]


class BatchIO(ctypes.Structure):
    _fields_ = [("seq", vp), ("offsets", vp), ("hash", vp), ("pos", vp), ("pick_offsets", vp), ("count", vp),
                ("capacity", u64), ("max_reads", u64), ("max_bases", u64), ("path", i32),
                ("tuned_ms", ctypes.c_float * 3)]


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _build.LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"the CUDA library {p} is not built; run paper_1811_10074_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _check(status: int):
    if status != SWS_OK:
        raise SwsError(status, load().sws_last_error().decode())


class Context:
    """An sws context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = vp()
        _check(load().sws_create(ctypes.byref(h), self.device))
        self.handle = h

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.sws_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nbytes: int):
        _check(load().sws_reserve(self.handle, int(nbytes)))

    def sync(self, stream=None):
        _check(load().sws_sync(self.handle, _stream(stream)))


def default_context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    with _lock:
        c = _ctx.get(device)
    if c is None:
        c = Context(device)
        with _lock:
            _ctx[device] = c
    return c


def _stream(stream):
    if stream is None:
        return vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return vp(stream.cuda_stream)
    return vp(int(stream))


def _ptr(t):
    return vp(t.data_ptr()) if t is not None else vp(0)


def _dev(t: torch.Tensor, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


# ------------------------------------------------------------------------------------------
# Entry points
# ------------------------------------------------------------------------------------------

def sliding_sum(op: str, w: int, x: torch.Tensor, out: torch.Tensor | None = None, variant: str = "auto",
                ctx: Context | None = None, stream=None) -> torch.Tensor:
    """Eq. 2 over ``x`` (int32 for the integer ops, float32 for add_f32, int32 [n, 2] for affine)."""
    _dev(x, "x")
    ctx = ctx or default_context(x.device.index)
    n = x.shape[0]
    m = max(n - w + 1, 0)
    if out is None:
        out = torch.empty((m,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    _dev(out, "out")
    _check(load().sws_sliding_sum(ctx.handle, OPS[op], int(w), _ptr(x), _ptr(out), n, VARIANTS[variant],
                                  _stream(stream)))
    return out


def tune_sliding_sum(op: str, w: int, n: int, ctx: Context | None = None, stream=None):
    """Time every variant that applies to (op, w) on n scratch elements; the context then uses the
    fastest for ``variant="auto"``.  Returns (chosen variant name, {variant name: ms})."""
    ctx = ctx or default_context(torch.cuda.current_device())
    chosen = ctypes.c_int(-1)
    ms = (ctypes.c_float * len(VARIANTS))()
    _check(load().sws_tune_sliding_sum(ctx.handle, OPS[op], int(w), int(n), ctypes.byref(chosen), ms, _stream(stream)))
    names = {v: k for k, v in VARIANTS.items()}
    return names[chosen.value], {names[i]: round(ms[i], 4) for i in range(len(VARIANTS)) if ms[i] >= 0}


def selftest_wait_timeout(which: str = "lookback", ctx: Context | None = None, stream=None) -> None:
    """Queue a bounded device wait on a flag nothing sets ("lookback" or "mbarrier"); the next
    ``Context.sync`` raises SwsError(TIMEOUT)."""
    ctx = ctx or default_context(torch.cuda.current_device())
    _check(load().sws_selftest_wait_timeout(ctx.handle, {"lookback": 0, "mbarrier": 1}[which], _stream(stream)))


def selftest_minimizer_timeout(ctx: Context | None = None, stream=None) -> torch.Tensor:
    """Queue the look-back minimizer kernel with its input copies withheld; returns the device
    count word (it must stay all ones) -- the next ``Context.sync`` raises SwsError(TIMEOUT)."""
    ctx = ctx or default_context(torch.cuda.current_device())
    cnt = torch.zeros(1, dtype=torch.int64, device=torch.device("cuda", ctx.device))
    _check(load().sws_selftest_minimizer_timeout(ctx.handle, _ptr(cnt), _stream(stream)))
    return cnt


def kmers(seq: torch.Tensor, n: int, k: int, kind: str = "hash", out: torch.Tensor | None = None,
          ctx: Context | None = None, stream=None) -> torch.Tensor:
    """k-mer values (int32 bit patterns when 2k <= 32, else int64)."""
    _dev(seq, "seq")
    ctx = ctx or default_context(seq.device.index)
    m = max(n - k + 1, 0)
    if out is None:
        out = torch.empty(m, dtype=torch.int32 if 2 * k <= 32 else torch.int64, device=seq.device)
    _check(load().sws_kmers(ctx.handle, _ptr(seq), int(n), int(k), KMER_KINDS[kind], _ptr(out), _stream(stream)))
    return out


def _trim(hash_out, pos_out, count, capacity, ctx, stream):
    ctx.sync(stream)
    c = int(count.item())
    if c > capacity:
        raise SwsError(SWS_ERR_CAPACITY, f"{c} picks exceed the capacity {capacity}")
    return hash_out[:c], pos_out[:c], c


def minimizers(seq: torch.Tensor, n: int, k: int, w: int, mode: str = "hash", nblocks: torch.Tensor | None = None,
               capacity: int | None = None, ctx: Context | None = None, stream=None, sync: bool = True):
    """(keys, positions) of the deduplicated minimizers; keys int32 bit patterns (2k <= 32) or int64.

    With ``sync=False`` returns the untrimmed buffers and the device count tensor."""
    _dev(seq, "seq")
    ctx = ctx or default_context(seq.device.index)
    dev = seq.device
    nwin = max(n - (w + k - 1) + 1, 0)
    if capacity is None:
        capacity = nwin
    h = torch.empty(max(capacity, 1), dtype=torch.int32 if 2 * k <= 32 else torch.int64, device=dev)
    p = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    nb = 0
    if nblocks is not None:
        _dev(nblocks, "nblocks")
        nb = nblocks.shape[0]
    _check(load().sws_minimizers(ctx.handle, _ptr(seq), int(n), int(k), int(w), MINI_MODES[mode],
                                 _ptr(nblocks) if nb else vp(0), nb, _ptr(h), _ptr(p), capacity, _ptr(cnt),
                                 _stream(stream)))
    if not sync:
        return h, p, cnt
    h, p, _ = _trim(h, p, cnt, capacity, ctx, stream)
    return h, p


def minimizers_count(seq: torch.Tensor, n: int, k: int, w: int, mode: str = "hash",
                     nblocks: torch.Tensor | None = None, ctx: Context | None = None, stream=None,
                     sync: bool = True):
    """Exact number of picks :func:`minimizers` would return (an int; with ``sync=False`` the
    device count tensor)."""
    _dev(seq, "seq")
    ctx = ctx or default_context(seq.device.index)
    cnt = torch.empty(1, dtype=torch.int64, device=seq.device)
    nb = 0
    if nblocks is not None:
        _dev(nblocks, "nblocks")
        nb = nblocks.shape[0]
    _check(load().sws_minimizers_count(ctx.handle, _ptr(seq), int(n), int(k), int(w), MINI_MODES[mode],
                                       _ptr(nblocks) if nb else vp(0), nb, _ptr(cnt), _stream(stream)))
    if not sync:
        return cnt
    ctx.sync(stream)
    return int(cnt.item())


def build_table(seq: torch.Tensor, n: int, k: int, w: int, bucket_bits: int, mode: str = "hash",
                nblocks: torch.Tensor | None = None, capacity: int | None = None, ctx: Context | None = None,
                stream=None):
    """Minimizers, then the seed table, in one call: (sorted keys, sorted positions, bucket offsets
    [2^bucket_bits + 1]).  Without a capacity, :func:`minimizers_count` sizes the outputs."""
    _dev(seq, "seq")
    ctx = ctx or default_context(seq.device.index)
    if capacity is None:
        capacity = minimizers_count(seq, n, k, w, mode, nblocks, ctx=ctx, stream=stream)
    dev = seq.device
    sh = torch.empty(max(capacity, 1), dtype=torch.int32 if 2 * k <= 32 else torch.int64, device=dev)
    sp = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    off = torch.empty((1 << bucket_bits) + 1, dtype=torch.int64, device=dev)
    nb = 0
    if nblocks is not None:
        _dev(nblocks, "nblocks")
        nb = nblocks.shape[0]
    m = u64()
    _check(load().sws_build_table(ctx.handle, _ptr(seq), int(n), int(k), int(w), MINI_MODES[mode],
                                  _ptr(nblocks) if nb else vp(0), nb, int(bucket_bits), _ptr(sh), _ptr(sp), capacity,
                                  _ptr(off), ctypes.byref(m), _stream(stream)))
    c = int(m.value)
    return sh[:c], sp[:c], off


def minimizers_from_keys(keys: torch.Tensor, w: int, capacity: int | None = None, ctx: Context | None = None,
                         stream=None, sync: bool = True):
    """Deduplicated sliding minimum (value, position) over a precomputed uint32 key array."""
    _dev(keys, "keys")
    ctx = ctx or default_context(keys.device.index)
    m = keys.shape[0]
    if capacity is None:
        capacity = max(m - w + 1, 0)
    h = torch.empty(max(capacity, 1), dtype=torch.int32, device=keys.device)
    p = torch.empty(max(capacity, 1), dtype=torch.int32, device=keys.device)
    cnt = torch.empty(1, dtype=torch.int64, device=keys.device)
    _check(load().sws_minimizers_from_keys(ctx.handle, _ptr(keys), m, int(w), _ptr(h), _ptr(p), capacity, _ptr(cnt),
                                           _stream(stream)))
    if not sync:
        return h, p, cnt
    h, p, _ = _trim(h, p, cnt, capacity, ctx, stream)
    return h, p


def minimizers_batch(seq: torch.Tensor, offsets: torch.Tensor, total_bases: int, k: int, w: int, mode: str = "hash",
                     capacity: int | None = None, ctx: Context | None = None, stream=None, sync: bool = True):
    """Per-read minimizers of reads stored back to back: (keys, read-local positions, pick offsets)."""
    _dev(seq, "seq")
    _dev(offsets, "offsets")
    ctx = ctx or default_context(seq.device.index)
    nreads = offsets.shape[0] - 1
    if capacity is None:
        capacity = max(int(total_bases), 1)
    dev = seq.device
    h = torch.empty(max(capacity, 1), dtype=torch.int32 if 2 * k <= 32 else torch.int64, device=dev)
    p = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    po = torch.empty(nreads + 1, dtype=torch.int64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    _check(load().sws_minimizers_batch(ctx.handle, _ptr(seq), _ptr(offsets), nreads, int(total_bases), int(k), int(w),
                                       MINI_MODES[mode], _ptr(h), _ptr(p), capacity, _ptr(po), _ptr(cnt),
                                       _stream(stream)))
    if not sync:
        return h, p, po, cnt
    h, p, _ = _trim(h, p, cnt, capacity, ctx, stream)
    return h, p, po


def kmer_table(hashes: torch.Tensor, pos: torch.Tensor, hash_bits: int, bucket_bits: int,
               ctx: Context | None = None, stream=None):
    """Seed table: (sorted hashes, sorted positions, bucket offsets [2^bucket_bits + 1])."""
    _dev(hashes, "hashes")
    _dev(pos, "pos")
    ctx = ctx or default_context(hashes.device.index)
    m = hashes.shape[0]
    sh = torch.empty_like(hashes)
    sp = torch.empty_like(pos)
    off = torch.empty((1 << bucket_bits) + 1, dtype=torch.int64, device=hashes.device)
    _check(load().sws_kmer_table(ctx.handle, _ptr(hashes), _ptr(pos), m, int(hash_bits), int(bucket_bits), _ptr(sh),
                                 _ptr(sp), _ptr(off), _stream(stream)))
    return sh, sp, off


class _DevArray:
    """A view of library-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


BATCH_OPTIONS = {"default": 0, "tune": 1, "lookback": 2}


class Batch:
    """A reusable batched-minimizer pipeline replayed as one CUDA graph (sws_batch_*)."""

    def __init__(self, max_reads: int, max_bases: int, k: int, w: int, mode: str = "hash", options: str = "default",
                 ctx: Context | None = None):
        self.ctx = ctx or default_context()
        h = vp()
        _check(load().sws_batch_create(self.ctx.handle, int(max_reads), int(max_bases), int(k), int(w),
                                       MINI_MODES[mode], BATCH_OPTIONS[options], ctypes.byref(h)))
        self.handle = h
        io = BatchIO()
        _check(load().sws_batch_io_get(self.handle, ctypes.byref(io)))
        self.io = io
        self.k = k
        dev = torch.device("cuda", self.ctx.device)
        hs = "<u4" if 2 * k <= 32 else "<u8"
        self.seq = torch.as_tensor(_DevArray(io.seq, ((int(max_bases) + 3) // 4,), "|u1"), device=dev)
        self.offsets = torch.as_tensor(_DevArray(io.offsets, (int(max_reads) + 1,), "<i8"), device=dev)
        self.hash = torch.as_tensor(_DevArray(io.hash, (int(io.capacity),), hs.replace("u", "i")), device=dev)
        self.pos = torch.as_tensor(_DevArray(io.pos, (int(io.capacity),), "<i4"), device=dev)
        self.pick_offsets = torch.as_tensor(_DevArray(io.pick_offsets, (int(max_reads) + 1,), "<i8"), device=dev)
        self.count = torch.as_tensor(_DevArray(io.count, (1,), "<i8"), device=dev)
        self.path = int(io.path)
        self.tuned_ms = tuple(float(v) for v in io.tuned_ms)
        self.nreads = 0

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.sws_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, seq: torch.Tensor, offsets: torch.Tensor, stream=None):
        """Copy packed reads and their offsets (device or host tensors) into the batch buffers."""
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.seq[: seq.numel()].copy_(seq, non_blocking=True)
            self.offsets[: offsets.numel()].copy_(offsets, non_blocking=True)

    def run(self, nreads: int, total_bases: int, stream=None):
        _check(load().sws_batch_run(self.handle, int(nreads), int(total_bases), _stream(stream)))
        self.nreads = int(nreads)

    def results(self):
        """(keys, positions, pick offsets) of the last run (waits for it)."""
        _check(load().sws_batch_sync(self.handle))
        c = int(self.count.item())
        return self.hash[:c], self.pos[:c], self.pick_offsets[: self.nreads + 1]


class Server:
    """Minimizer server with continuous batching (sws_server_*).  Requests are host sequences."""

    def __init__(self, k: int, w: int, slots: int = 4, max_requests_per_batch: int = 256,
                 max_bases_per_batch: int = 1 << 22, hbm_budget_bytes: int = 0, mode: str = "hash",
                 ctx: Context | None = None):
        import numpy as np  # noqa: F401  (results are numpy arrays)
        self.ctx = ctx or default_context()
        cfg = ServerConfig(k, w, MINI_MODES[mode], slots, max_requests_per_batch, max_bases_per_batch,
                           hbm_budget_bytes)
        h = vp()
        _check(load().sws_server_create(self.ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self.w = w

    def submit(self, packed, nbases: int) -> int:
        """Queue one packed sequence (numpy uint8 array or CPU tensor); returns the request id."""
        import numpy as np
        arr = packed.numpy() if hasattr(packed, "numpy") else packed
        arr = np.ascontiguousarray(arr, dtype=np.uint8)
        rid = u64()
        _check(load().sws_server_submit(self.handle, vp(arr.ctypes.data), int(nbases), ctypes.byref(rid)))
        return int(rid.value)

    def submit_many(self, requests) -> list:
        """Queue many (packed, nbases) requests in one call; returns their ids in order."""
        import numpy as np
        arrs = [np.ascontiguousarray(p.numpy() if hasattr(p, "numpy") else p, dtype=np.uint8) for p, _ in requests]
        count = len(arrs)
        ptrs = (vp * max(count, 1))(*[a.ctypes.data for a in arrs])
        ns = (u64 * max(count, 1))(*[int(nb) for _, nb in requests])
        ids = (u64 * max(count, 1))()
        _check(load().sws_server_submit_batch(self.handle, ptrs, ns, count, ids))
        return [int(ids[i]) for i in range(count)]

    def wait(self, rid: int, timeout: float = 60.0) -> bool:
        done = i32()
        _check(load().sws_server_wait(self.handle, int(rid), float(timeout), ctypes.byref(done)))
        return bool(done.value)

    def result(self, rid: int, capacity: int | None = None):
        """(keys uint32, positions uint32, latency seconds) of an answered request."""
        import numpy as np
        cap = capacity if capacity is not None else 1 << 16
        while True:
            h = np.empty(max(cap, 1), dtype=np.uint32)
            p = np.empty(max(cap, 1), dtype=np.uint32)
            cnt = u64()
            lat = ctypes.c_double()
            st = load().sws_server_result(self.handle, int(rid), vp(h.ctypes.data), vp(p.ctypes.data), cap,
                                          ctypes.byref(cnt), ctypes.byref(lat))
            if st == SWS_ERR_CAPACITY and cnt.value > cap:
                cap = int(cnt.value)
                continue
            _check(st)
            c = int(cnt.value)
            return h[:c], p[:c], float(lat.value)

    def collect_raw(self, max_n: int = 4096, timeout: float = 0.0):
        """Collect up to max_n answered requests: numpy arrays (ids, counts, latencies seconds,
        key pointers, position pointers).  The answers stay in the server's pinned memory until
        :meth:`release`; :meth:`views` turns one pair of pointers into arrays."""
        import numpy as np
        ids = np.empty(max(max_n, 1), dtype=np.uint64)
        cnt = np.empty(max(max_n, 1), dtype=np.uint64)
        lat = np.empty(max(max_n, 1), dtype=np.float64)
        hp = np.empty(max(max_n, 1), dtype=np.uint64)
        pp = np.empty(max(max_n, 1), dtype=np.uint64)
        n = u64()
        _check(load().sws_server_collect(self.handle, int(max_n), float(timeout), vp(ids.ctypes.data),
                                         vp(cnt.ctypes.data), vp(hp.ctypes.data), vp(pp.ctypes.data),
                                         vp(lat.ctypes.data), ctypes.byref(n)))
        k = int(n.value)
        return ids[:k], cnt[:k], lat[:k], hp[:k], pp[:k]

    @staticmethod
    def views(count: int, hash_ptr: int, pos_ptr: int):
        """(keys, positions) uint32 arrays over a collected answer's pinned memory (no copy)."""
        import numpy as np
        if count == 0:
            return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
        ht = ctypes.cast(int(hash_ptr), ctypes.POINTER(ctypes.c_uint32))
        pt = ctypes.cast(int(pos_ptr), ctypes.POINTER(ctypes.c_uint32))
        return np.ctypeslib.as_array(ht, shape=(int(count),)), np.ctypeslib.as_array(pt, shape=(int(count),))

    def release(self, ids):
        """Forget collected (or uncollected, answered) requests and free their result memory."""
        import numpy as np
        a = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
        _check(load().sws_server_release(self.handle, vp(a.ctypes.data), a.size))

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().sws_server_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(load().sws_server_reset_stats(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.sws_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def seed_lookup(sorted_hash: torch.Tensor, offsets: torch.Tensor, hash_bits: int, bucket_bits: int,
                query_hash: torch.Tensor, ctx: Context | None = None, stream=None):
    """(first int64, count int32) of each query seed's run in a table from :func:`kmer_table`."""
    _dev(sorted_hash, "sorted_hash")
    _dev(query_hash, "query_hash")
    ctx = ctx or default_context(query_hash.device.index)
    nq = query_hash.shape[0]
    first = torch.empty(max(nq, 1), dtype=torch.int64, device=query_hash.device)
    count = torch.empty(max(nq, 1), dtype=torch.int32, device=query_hash.device)
    _check(load().sws_seed_lookup(ctx.handle, _ptr(sorted_hash), sorted_hash.shape[0], int(hash_bits), int(bucket_bits),
                                  _ptr(offsets), _ptr(query_hash), nq, _ptr(first), _ptr(count), _stream(stream)))
    return first[:nq], count[:nq]


def seed_hits(first: torch.Tensor, count: torch.Tensor, sorted_pos: torch.Tensor, max_occ: int = 0,
              capacity: int | None = None, ctx: Context | None = None, stream=None, sync: bool = True):
    """(hit_query, hit_pos) pairs of the runs from :func:`seed_lookup` (seeds with more than
    max_occ hits skipped).  With ``sync=False`` returns the untrimmed buffers and the count."""
    _dev(first, "first")
    ctx = ctx or default_context(first.device.index)
    nq = first.shape[0]
    if capacity is None:
        capacity = int(count.to(torch.int64).sum().item()) if nq else 0
    hq = torch.empty(max(capacity, 1), dtype=torch.int32, device=first.device)
    hp = torch.empty(max(capacity, 1), dtype=torch.int32, device=first.device)
    cnt = torch.empty(1, dtype=torch.int64, device=first.device)
    if sorted_pos.numel() == 0:  # an empty table: every count is 0, the array is never read
        sorted_pos = torch.zeros(1, dtype=torch.int32, device=first.device)
    _check(load().sws_seed_hits(ctx.handle, _ptr(first), _ptr(count), nq, int(max_occ) & 0xFFFFFFFF, _ptr(sorted_pos),
                                _ptr(hq), _ptr(hp), capacity, _ptr(cnt), _stream(stream)))
    if not sync:
        return hq, hp, cnt
    ctx.sync(stream)
    c = int(cnt.item())
    if c > capacity:
        raise SwsError(SWS_ERR_CAPACITY, f"{c} hits exceed the capacity {capacity}")
    return hq[:c], hp[:c]


def minimizer_strands(seq: torch.Tensor, n: int, k: int, pos: torch.Tensor, base_offsets: torch.Tensor | None = None,
                      pick_offsets: torch.Tensor | None = None, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """uint8 strand of each pick: 0 forward (or palindrome), 1 reverse complement, 255 outside."""
    _dev(seq, "seq")
    ctx = ctx or default_context(seq.device.index)
    m = pos.shape[0]
    out = torch.empty(max(m, 1), dtype=torch.uint8, device=seq.device)
    nreads = base_offsets.shape[0] - 1 if base_offsets is not None else 0
    _check(load().sws_minimizer_strands(ctx.handle, _ptr(seq), int(n), int(k),
                                        _ptr(base_offsets) if base_offsets is not None else vp(0),
                                        _ptr(pick_offsets) if pick_offsets is not None else vp(0), nreads, _ptr(pos), m,
                                        _ptr(out), _stream(stream)))
    return out[:m]
