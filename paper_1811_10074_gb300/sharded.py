"""The seed table of a genome sharded over several processes (one per GPU): Sec. 2.4's table built
from the minimizers of the whole sequence, each rank owning one range of hash values.

Steps, per rank r of R (R a power of two):

1. Windows.  The genome's windows are split into R contiguous ranges starting at multiples of 4
   bases (byte boundaries of the 2-bit packing); rank r holds the bases its windows cover (its
   range plus the w + k - 2 bases after it) and computes their minimizers with global positions.
2. Seams.  A rank's first window always stores its pick; where that pick is the previous rank's
   last pick (the same position: positions strictly increase), it is dropped.  The ranks' last
   pick positions are exchanged with one all-gather of R integers.
3. Exchange.  Hit (h, p) belongs to rank h >> (hash_bits - log2 R); each rank sends every other
   rank its hits for that rank's range (point-to-point sends and receives, so the same code runs
   on NCCL and on gloo), after an all-gather of the R x R counts.  Hits arrive from ranks in rank
   order, hence in position order.
4. Local table.  Each rank sorts its hits by hash (stable: positions stay ascending) and builds the
   pointer table of the buckets in its range; its offsets are shifted by the number of hits of
   the ranks before it, so the ranks' shards, concatenated in rank order, are exactly the table
   of the whole genome.

Only step 1 and step 4 compute; they run through the CUDA library by default (``minimizers`` and
``kmer_table`` of the binding on the rank's device).  Other implementations of the same two calls
can be passed in (the tests pass the CPU reference to check the exchange logic on gloo ranks).
"""

from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def window_ranges(n: int, k: int, w: int, world: int):
    """Per rank: (first window, end window, first base, end base) of its share of the windows of
    an n-base sequence; windows start at multiples of 4 bases."""
    nwin = max(n - (w + k - 1) + 1, 0)
    bounds = [(nwin * r // world) // 4 * 4 for r in range(world)] + [nwin]
    out = []
    for r in range(world):
        w0, w1 = bounds[r], bounds[r + 1]
        if w1 <= w0:
            out.append((w0, w0, w0, w0))
        else:
            out.append((w0, w1, w0, min(n, w1 + w + k - 2)))
    return out


def _clip_nblocks(nblocks: np.ndarray | None, b0: int, b1: int) -> np.ndarray:
    if nblocks is None or len(nblocks) == 0:
        return np.zeros((0, 2), dtype=np.int64)
    nb = np.asarray(nblocks, dtype=np.int64).reshape(-1, 2)
    nb = nb[(nb[:, 1] > b0) & (nb[:, 0] < b1)]
    return np.clip(nb - b0, 0, b1 - b0).astype(np.int64)


def _device_minimizers(device):
    from . import binding as B

    def fn(seq_bytes: np.ndarray, n: int, k: int, w: int, mode: str, nblocks: np.ndarray):
        seq = torch.from_numpy(np.ascontiguousarray(seq_bytes)).to(device)
        nb = torch.from_numpy(nblocks).to(device) if len(nblocks) else None
        h, p = B.minimizers(seq, n, k, w, mode=mode, nblocks=nb)
        hv = h.cpu().numpy()
        hv = hv.view(np.uint32).astype(np.uint64) if hv.dtype == np.int32 else hv.view(np.uint64)
        return hv, p.cpu().numpy().view(np.uint32)
    return fn


def _device_table(device):
    from . import binding as B

    def fn(hashes: np.ndarray, pos: np.ndarray, hash_bits: int, bucket_bits: int):
        if hash_bits <= 32:
            hd = torch.from_numpy(hashes.astype(np.uint32).view(np.int32)).to(device)
        else:
            hd = torch.from_numpy(hashes.astype(np.uint64).view(np.int64)).to(device)
        pd = torch.from_numpy(pos.astype(np.uint32).view(np.int32)).to(device)
        sh, sp, off = B.kmer_table(hd, pd, hash_bits, bucket_bits)
        shv = sh.cpu().numpy()
        shv = shv.view(np.uint32).astype(np.uint64) if shv.dtype == np.int32 else shv.view(np.uint64)
        return shv, sp.cpu().numpy().view(np.uint32), off.cpu().numpy().view(np.uint64)
    return fn


def sharded_seed_table(local_seq, n: int, k: int, w: int, bucket_bits: int, nblocks=None, mode: str = "hash",
                       group=None, device=None, minimizers_fn=None, table_fn=None):
    """This rank's shard of the seed table of an n-base genome (call on every rank of `group`).

    local_seq   : the packed bytes of this rank's bases, window_ranges(n, k, w, R)[rank][2:] (the
                  first base is a multiple of 4, so the bytes are a plain slice of the genome's).
    nblocks     : the genome's N-blocks, global half-open base intervals (int64 [m][2]) or None.
    bucket_bits : pointer-table buckets of the whole table are 2^bucket_bits; R <= 2^bucket_bits.
    Returns (sorted_hash uint64, sorted_pos uint32, offsets uint64, (first bucket, end bucket),
    hits before this shard): offsets[i] is the global index of the first hit of bucket
    first + i, for i = 0 .. end - first (the last entry is where the next shard begins).
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if world & (world - 1):
        raise ValueError("the number of ranks must be a power of two")
    hash_bits = 2 * k
    rbits = world.bit_length() - 1
    if bucket_bits < rbits or bucket_bits > min(hash_bits, 32):
        raise ValueError("need log2(ranks) <= bucket_bits <= min(2k, 32)")
    if device is None and torch.cuda.is_available():
        device = torch.device("cuda", torch.cuda.current_device())
    minimizers_fn = minimizers_fn or _device_minimizers(device)
    table_fn = table_fn or _device_table(device)
    backend = dist.get_backend(group)
    comm = device if backend == "nccl" else torch.device("cpu")

    # 1. the minimizers of this rank's windows, at global positions
    w0, w1, b0, b1 = window_ranges(n, k, w, world)[rank]
    if b1 > b0:
        h, p = minimizers_fn(np.asarray(local_seq, dtype=np.uint8), b1 - b0, k, w, mode,
                             _clip_nblocks(nblocks, b0, b1))
        h = np.asarray(h, dtype=np.uint64)
        p = np.asarray(p, dtype=np.uint64) + np.uint64(b0)
    else:
        h = np.zeros(0, np.uint64)
        p = np.zeros(0, np.uint64)

    # 2. the seam: this rank's first pick may be the last pick of the ranks before it
    last = torch.tensor([int(p[-1]) if p.size else -1], dtype=torch.int64, device=comm)
    lasts = [torch.zeros(1, dtype=torch.int64, device=comm) for _ in range(world)]
    dist.all_gather(lasts, last, group=group)
    prev = max([int(x.item()) for x in lasts[:rank]], default=-1)
    if p.size and int(p[0]) == prev:
        h, p = h[1:], p[1:]

    # 3. every hit to the rank owning its hash range
    dest = (h >> np.uint64(hash_bits - rbits)).astype(np.int64) if rbits else np.zeros(h.size, np.int64)
    order = np.argsort(dest, kind="stable")  # position order within each destination
    h, p, dest = h[order], p[order], dest[order]
    counts = np.bincount(dest, minlength=world).astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)])
    mine = torch.from_numpy(counts).to(comm)
    allc = [torch.zeros(world, dtype=torch.int64, device=comm) for _ in range(world)]
    dist.all_gather(allc, mine, group=group)
    cm = np.stack([c.cpu().numpy() for c in allc])  # cm[src][dst]
    pairs = np.stack([h.view(np.int64), p.astype(np.int64)], axis=1) if h.size else np.zeros((0, 2), np.int64)
    recv = {}
    ops = []
    for q in range(world):
        if q == rank:
            continue
        if cm[rank][q]:
            t = torch.from_numpy(np.ascontiguousarray(pairs[starts[q]:starts[q + 1]])).to(comm)
            ops.append(dist.isend(t, dst=q, group=group))
        if cm[q][rank]:
            buf = torch.empty((int(cm[q][rank]), 2), dtype=torch.int64, device=comm)
            recv[q] = buf
            ops.append(dist.irecv(buf, src=q, group=group))
    for op in ops:
        op.wait()
    parts = []
    for q in range(world):
        if q == rank:
            parts.append(pairs[starts[rank]:starts[rank + 1]])
        elif q in recv:
            parts.append(recv[q].cpu().numpy())
    got = np.concatenate(parts) if parts else np.zeros((0, 2), np.int64)
    H = got[:, 0].view(np.uint64).copy()
    Pp = got[:, 1].astype(np.uint32)

    # 4. the local table, its buckets shifted to global hit indices
    per_rank = cm.sum(axis=0)  # hits each rank owns
    before = int(per_rank[:rank].sum())
    sh, sp, off_full = table_fn(H, Pp, hash_bits, bucket_bits)
    nb = 1 << bucket_bits
    bl, bh = rank * (nb // world), (rank + 1) * (nb // world)
    off = np.asarray(off_full, dtype=np.uint64)[bl:bh + 1] + np.uint64(before)
    return np.asarray(sh, dtype=np.uint64), np.asarray(sp, dtype=np.uint32), off, (bl, bh), before
