"""Python access to the plain CPU oracle in ``sws_oracle.c``.

TEST INFRASTRUCTURE.  The oracle states what the sliding-window-sum library computes
(Eq. 2, the k-mer / minimizer definitions of Sec. 2.4 and the seed table) as slowly and
plainly as possible.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import it; the library itself never does.  It shares no code with the
CUDA path: this wrapper passes numpy arrays to the C functions and nothing else.

The shared object is compiled with gcc on first use (or by :func:`build`) into
``oracle/_build``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sws_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libsws_oracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"add_i32": 0, "min_i32": 1, "max_i32": 2, "xor_i32": 3, "affine_u32": 4, "add_f32": 5}
KMER_KINDS = {"fwd": 0, "rc": 1, "canonical": 2, "hash": 3}
MINI_MODES = {"hash": 0, "canonical": 1, "fwd": 2}

u64 = ctypes.c_uint64
i32 = ctypes.c_int
vp = ctypes.c_void_p


def build(force: bool = False, extra_flags=(), src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, *extra_flags]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building if needed) and declare the oracle's C functions."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        p = path or build()
        lib = ctypes.CDLL(p)
        lib.oracle_sliding_sum.restype = u64
        lib.oracle_sliding_sum.argtypes = [i32, i32, vp, u64, vp]
        lib.oracle_sliding_sum_at.restype = None
        lib.oracle_sliding_sum_at.argtypes = [i32, i32, vp, u64, vp, u64, vp]
        lib.oracle_hash.restype = u64
        lib.oracle_hash.argtypes = [u64, i32]
        lib.oracle_hash_inv.restype = u64
        lib.oracle_hash_inv.argtypes = [u64, i32]
        lib.oracle_hash_is_bijection.restype = i32
        lib.oracle_hash_is_bijection.argtypes = [i32]
        lib.oracle_kmers.restype = u64
        lib.oracle_kmers.argtypes = [vp, u64, i32, i32, vp]
        lib.oracle_minimizers.restype = u64
        lib.oracle_minimizers.argtypes = [vp, u64, i32, i32, i32, vp, u64, vp, vp, u64, i32]
        lib.oracle_minimizers_batch.restype = u64
        lib.oracle_minimizers_batch.argtypes = [vp, vp, u64, i32, i32, i32, vp, vp, u64, vp]
        lib.oracle_minimizers_from_keys.restype = u64
        lib.oracle_minimizers_from_keys.argtypes = [vp, u64, i32, vp, vp, u64]
        lib.oracle_minimizers_from_keys_deque.restype = u64
        lib.oracle_minimizers_from_keys_deque.argtypes = [vp, u64, i32, vp, vp, u64]
        lib.oracle_kmer_table.restype = i32
        lib.oracle_kmer_table.argtypes = [vp, vp, u64, i32, i32, vp, vp, vp]
        lib.oracle_strands.restype = None
        lib.oracle_strands.argtypes = [vp, u64, i32, vp, vp, u64, vp, u64, vp]
        lib.oracle_seed_hits.restype = u64
        lib.oracle_seed_hits.argtypes = [vp, vp, u64, vp, u64, ctypes.c_uint32, vp, vp, vp, u64]
        if path is None:
            _lib = lib
        return lib


def _np(a, dtype=None):
    """torch tensor or array-like -> contiguous numpy array (on the CPU)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a)
    if dtype is not None and a.dtype != dtype:
        a = a.view(dtype) if a.dtype.itemsize == np.dtype(dtype).itemsize else a.astype(dtype)
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _elem_view(op: str, x) -> np.ndarray:
    x = _np(x)
    if op == "affine_u32":
        return np.ascontiguousarray(x.reshape(-1).view(np.uint32).reshape(-1, 2))
    if op == "add_f32":
        return x.astype(np.float32, copy=False).reshape(-1)
    return x.reshape(-1).view(np.int32) if x.dtype.itemsize == 4 else x.astype(np.int32).reshape(-1)


def _out_array(op: str, m: int) -> np.ndarray:
    if op == "affine_u32":
        return np.zeros((m, 2), dtype=np.uint32)
    if op == "add_f32":
        return np.zeros(m, dtype=np.float64)
    return np.zeros(m, dtype=np.int32)


def sliding_sum(op: str, w: int, x, lib=None) -> np.ndarray:
    """Eq. 2 over the whole input: ``n - w + 1`` outputs (int32 bit patterns, uint32 pairs for
    affine, float64 for fp32 add)."""
    lib = lib or load()
    xv = _elem_view(op, x)
    n = xv.shape[0]
    m = max(n - w + 1, 0) if w >= 1 else 0
    y = _out_array(op, max(m, 1))
    got = lib.oracle_sliding_sum(OPS[op], w, _ptr(xv), n, _ptr(y))
    assert got == m
    return y[:m]


def sliding_sum_at(op: str, w: int, x, idx, lib=None) -> np.ndarray:
    """Eq. 2 at the output indices ``idx`` only."""
    lib = lib or load()
    xv = _elem_view(op, x)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    n = xv.shape[0]
    assert idx.size == 0 or int(idx.max()) + w <= n
    y = _out_array(op, max(idx.size, 1))
    lib.oracle_sliding_sum_at(OPS[op], w, _ptr(xv), n, _ptr(idx), idx.size, _ptr(y))
    return y[: idx.size]


def hash64(x: int, bits: int, lib=None) -> int:
    return int((lib or load()).oracle_hash(x, bits))


def hash64_inv(h: int, bits: int, lib=None) -> int:
    return int((lib or load()).oracle_hash_inv(h, bits))


def hash_is_bijection(bits: int, lib=None) -> bool:
    r = (lib or load()).oracle_hash_is_bijection(bits)
    if r < 0:
        raise MemoryError("oracle bitmap allocation failed")
    return bool(r)


def kmers(seq, n: int, k: int, kind: str = "hash", lib=None) -> np.ndarray:
    """Values (uint64) of the ``n - k + 1`` k-mers of a packed sequence."""
    lib = lib or load()
    s = _np(seq, np.uint8)
    m = max(n - k + 1, 0)
    out = np.zeros(max(m, 1), dtype=np.uint64)
    got = lib.oracle_kmers(_ptr(s), n, k, KMER_KINDS[kind], _ptr(out))
    assert got == m
    return out[:m]


def minimizers(seq, n: int, k: int, w: int, mode: str = "hash", nblocks=None, deque: bool = False,
               cap: int | None = None, lib=None):
    """(keys uint64, positions uint32) of the deduplicated minimizers of a packed sequence."""
    lib = lib or load()
    s = _np(seq, np.uint8)
    nb = np.zeros((0, 2), dtype=np.int64) if nblocks is None else np.ascontiguousarray(np.asarray(nblocks, dtype=np.int64).reshape(-1, 2))
    if cap is None:
        cap = max(n - k - w + 2, 0) + 1
    h = np.zeros(max(cap, 1), dtype=np.uint64)
    p = np.zeros(max(cap, 1), dtype=np.uint32)
    cnt = lib.oracle_minimizers(_ptr(s), n, k, w, MINI_MODES[mode], _ptr(nb), nb.shape[0], _ptr(h), _ptr(p), cap,
                                1 if deque else 0)
    cnt = int(cnt)
    assert cnt <= cap
    return h[:cnt], p[:cnt]


def minimizers_batch(seq, offs, k: int, w: int, mode: str = "hash", lib=None):
    """Per-read minimizers of reads stored back to back: (keys, read-local positions, pick offsets)."""
    lib = lib or load()
    s = _np(seq, np.uint8)
    offs = np.ascontiguousarray(np.asarray(offs, dtype=np.int64))
    nreads = offs.size - 1
    cap = int(max(offs[-1], 1))
    h = np.zeros(cap, dtype=np.uint64)
    p = np.zeros(cap, dtype=np.uint32)
    po = np.zeros(nreads + 1, dtype=np.uint64)
    cnt = int(lib.oracle_minimizers_batch(_ptr(s), _ptr(offs), nreads, k, w, MINI_MODES[mode], _ptr(h), _ptr(p), cap,
                                          _ptr(po)))
    return h[:cnt], p[:cnt], po


def minimizers_from_keys(keys, w: int, deque: bool = False, lib=None):
    """Deduplicated (key, position) sliding minima over a precomputed key array (naive per-window
    scan, or with ``deque`` the queue-based scan)."""
    lib = lib or load()
    kv = _np(keys)
    if kv.dtype != np.uint64:
        kv = kv.view(np.uint32) if kv.dtype == np.int32 else kv
        kv = kv.astype(np.uint64)
    kv = np.ascontiguousarray(kv)
    m = kv.size
    cap = max(m - w + 1, 1)
    h = np.zeros(cap, dtype=np.uint64)
    p = np.zeros(cap, dtype=np.uint32)
    fn = lib.oracle_minimizers_from_keys_deque if deque else lib.oracle_minimizers_from_keys
    cnt = int(fn(_ptr(kv), m, w, _ptr(h), _ptr(p), cap))
    return h[:cnt], p[:cnt]


# ------------------------------------------------------------------------------------------
# Chunked multi-threaded drivers (for timing the oracle on all host cores).  They split the
# windows into contiguous ranges, run the plain oracle above on each range's inputs (the range
# plus the w - 1 (+ k - 1) elements its last windows reach) in a thread each -- ctypes releases
# the GIL during the C call -- and join the per-range picks in order.  A range's first window
# always stores its pick, so where that pick is the previous range's last pick (the same
# position: positions strictly increase) it is dropped once.  The arithmetic is the oracle's.
# ------------------------------------------------------------------------------------------

def _join_ranges(parts):
    hs, ps = [], []
    last = None
    for h, p in parts:
        if last is not None and p.size and int(p[0]) == last:
            h, p = h[1:], p[1:]
        if p.size:
            last = int(p[-1])
        hs.append(h)
        ps.append(p)
    if not hs:
        return np.zeros(0, np.uint64), np.zeros(0, np.uint32)
    return np.concatenate(hs), np.concatenate(ps)


def minimizers_from_keys_chunked(keys, w: int, threads: int, deque: bool = False, lib=None):
    """:func:`minimizers_from_keys` with the windows split over ``threads`` threads."""
    from concurrent.futures import ThreadPoolExecutor
    lib = lib or load()
    kv = _np(keys)
    if kv.dtype != np.uint64:
        kv = kv.view(np.uint32) if kv.dtype == np.int32 else kv
        kv = kv.astype(np.uint64)
    kv = np.ascontiguousarray(kv)
    m = kv.size
    nwin = max(m - w + 1, 0)
    threads = max(1, min(int(threads), max(nwin, 1)))
    bounds = [nwin * t // threads for t in range(threads + 1)]

    def one(t):
        p0, p1 = bounds[t], bounds[t + 1]
        if p1 <= p0:
            return np.zeros(0, np.uint64), np.zeros(0, np.uint32)
        h, p = minimizers_from_keys(kv[p0:p1 + w - 1], w, deque=deque, lib=lib)
        return h, (p.astype(np.uint64) + p0).astype(np.uint32)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, range(threads)))
    return _join_ranges(parts)


def minimizers_chunked(seq, n: int, k: int, w: int, threads: int, mode: str = "hash", deque: bool = False,
                       lib=None):
    """:func:`minimizers` of a packed sequence without N-blocks, the windows split over ``threads``
    threads (ranges start at multiples of 4 bases, i.e. at byte boundaries of the packing)."""
    from concurrent.futures import ThreadPoolExecutor
    lib = lib or load()
    s = _np(seq, np.uint8)
    nwin = max(n - (w + k - 1) + 1, 0)
    threads = max(1, min(int(threads), max(nwin // 4, 1)))
    bounds = [(nwin * t // threads) // 4 * 4 for t in range(threads)] + [nwin]

    def one(t):
        p0, p1 = bounds[t], bounds[t + 1]
        if p1 <= p0:
            return np.zeros(0, np.uint64), np.zeros(0, np.uint32)
        nb = p1 - p0 + w + k - 2  # bases the range's windows cover
        h, p = minimizers(s[p0 // 4:(p0 + nb + 3) // 4], nb, k, w, mode=mode, deque=deque, lib=lib)
        return h, (p.astype(np.uint64) + p0).astype(np.uint32)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, range(threads)))
    return _join_ranges(parts)


def kmer_table(hashes, pos, hash_bits: int, bucket_bits: int, lib=None):
    """(sorted hashes, sorted positions, bucket offsets of length 2^bucket_bits + 1)."""
    lib = lib or load()
    h = np.ascontiguousarray(_np(hashes).astype(np.uint64))
    p = np.ascontiguousarray(_np(pos).astype(np.uint32))
    m = h.size
    sh = np.zeros(max(m, 1), dtype=np.uint64)
    sp = np.zeros(max(m, 1), dtype=np.uint32)
    off = np.zeros((1 << bucket_bits) + 1, dtype=np.uint64)
    rc = lib.oracle_kmer_table(_ptr(h), _ptr(p), m, hash_bits, bucket_bits, _ptr(sh), _ptr(sp), _ptr(off))
    if rc != 0:
        raise ValueError("bad bucket_bits")
    return sh[:m], sp[:m], off


def seed_hits(ref_hash, ref_pos, query_hash, max_occ: int = 0, lib=None):
    """Seed hits (query index, reference position) of each query seed against the reference's
    (hash, position) seeds, seeds with more than max_occ hits skipped (0: no limit).
    Returns (count per query before the filter, hit_query, hit_pos)."""
    lib = lib or load()
    h = np.ascontiguousarray(_np(ref_hash).astype(np.uint64))
    p = np.ascontiguousarray(_np(ref_pos).astype(np.uint32))
    q = np.ascontiguousarray(_np(query_hash).astype(np.uint64))
    m, nq = h.size, q.size
    cnt = np.zeros(max(nq, 1), dtype=np.uint32)
    # first pass sizes the output
    total = int(lib.oracle_seed_hits(_ptr(h), _ptr(p), m, _ptr(q), nq, int(max_occ), _ptr(cnt), None, None, 0))
    hq = np.zeros(max(total, 1), dtype=np.uint32)
    hp = np.zeros(max(total, 1), dtype=np.uint32)
    got = int(lib.oracle_seed_hits(_ptr(h), _ptr(p), m, _ptr(q), nq, int(max_occ), _ptr(cnt), _ptr(hq), _ptr(hp), total))
    assert got == total
    return cnt[:nq], hq[:total], hp[:total]


def strands(seq, n: int, k: int, pos, offs=None, pick_offs=None, lib=None) -> np.ndarray:
    """Strand (0 forward / palindrome, 1 reverse complement, 255 outside) of each pick."""
    lib = lib or load()
    s = _np(seq, np.uint8)
    pv = np.ascontiguousarray(_np(pos).astype(np.uint32))
    m = pv.size
    out = np.zeros(max(m, 1), dtype=np.uint8)
    if offs is None:
        lib.oracle_strands(_ptr(s), n, k, None, None, 0, _ptr(pv), m, _ptr(out))
    else:
        o = np.ascontiguousarray(np.asarray(offs, dtype=np.int64))
        po = np.ascontiguousarray(np.asarray(pick_offs, dtype=np.uint64))
        lib.oracle_strands(_ptr(s), n, k, _ptr(o), _ptr(po), o.size - 1, _ptr(pv), m, _ptr(out))
    return out[:m]
