"""The sharded seed table on CPU gloo ranks (world size 2 and 4, one process per rank): each rank
computes the minimizers of its share of the windows and builds its shard after the exchange by
hash range; the shards concatenated in rank order must equal the oracle's table of the whole
genome.  The per-rank computation is the oracle here (the exchange logic is what is tested; on
GPUs the same two calls run through the CUDA library)."""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1811_10074_gb300 import sharded, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import numpy as np
import torch.distributed as dist
import oracle
from paper_1811_10074_gb300 import sharded
from test_sharded_table import make_genome
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
case = int(os.environ["CASE"])
seq, n, nb, k, w, bb, mode = make_genome(case)
w0, w1, b0, b1 = sharded.window_ranges(n, k, w, world)[rank]
local = seq[b0 // 4:(b1 + 3) // 4]
mini = lambda s, m, k_, w_, md, nbl: oracle.minimizers(s, m, k_, w_, mode=md, nblocks=nbl)
table = lambda h, p, hb, b: oracle.kmer_table(h, p, hb, b)
sh, sp, off, (bl, bh), before = sharded.sharded_seed_table(local, n, k, w, bb, nblocks=nb, mode=mode,
                                                           minimizers_fn=mini, table_fn=table)
np.savez(os.path.join(os.environ["OUT"], f"shard{rank}.npz"), sh=sh, sp=sp, off=off, bl=bl, bh=bh, before=before)
dist.barrier()
dist.destroy_process_group()
"""


def make_genome(case: int):
    """(packed bytes, n, N-blocks, k, w, bucket_bits, key mode) of a test case."""
    if case == 0:  # uniform bases with N-blocks, one across the middle (a chunk seam)
        n = 120_001
        seq = synth.acgt_uniform_packed(n, seed=5).numpy()
        nb = np.array([[1000, 1500], [59_990, 60_030], [90_000, 90_001], [119_990, 120_001]], dtype=np.int64)
        return seq, n, nb, 15, 10, 12, "hash"
    if case == 1:  # 38-bit hashes
        n = 80_003
        seq = synth.acgt_uniform_packed(n, seed=6).numpy()
        return seq, n, None, 19, 10, 14, "hash"
    # low complexity: long runs of equal k-mers, picks that span the seams
    n = 40_000
    codes = np.tile(np.array([0, 0, 1, 0, 0, 1, 2], dtype=np.uint8), n // 7 + 1)[:n]
    codes[17_000:23_000] = 3
    import torch
    seq = synth.pack_codes(torch.from_numpy(codes)).numpy()
    return seq, n, np.array([[30_000, 30_004]], dtype=np.int64), 5, 4, 6, "fwd"


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_sharded_table_equals_whole_genome_table(tmp_path, world, case):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", CASE=str(case),
                   OUT=str(tmp_path))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-3000:]
    shards = [np.load(tmp_path / f"shard{r}.npz") for r in range(world)]
    seq, n, nb, k, w, bb, mode = make_genome(case)
    mh, mp = oracle.minimizers(seq, n, k, w, mode=mode, nblocks=nb)
    rh, rp, ro = oracle.kmer_table(mh, mp, 2 * k, bb)
    assert np.array_equal(np.concatenate([s["sh"] for s in shards]), rh)
    assert np.array_equal(np.concatenate([s["sp"] for s in shards]), rp)
    # the pointer tables: each shard covers its bucket range; consecutive shards share an endpoint
    off = np.concatenate([shards[0]["off"]] + [s["off"][1:] for s in shards[1:]])
    assert np.array_equal(off, ro)
    assert [int(s["bl"]) for s in shards] == [r * ((1 << bb) // world) for r in range(world)]
    assert int(shards[-1]["off"][-1]) == mh.size


def test_window_ranges_cover_every_window_once():
    for n, k, w, world in ((1000, 15, 10, 4), (30, 15, 10, 2), (100_001, 19, 50, 8), (10, 3, 3, 4)):
        nwin = max(n - (w + k - 1) + 1, 0)
        rs = sharded.window_ranges(n, k, w, world)
        covered = []
        for w0, w1, b0, b1 in rs:
            assert w0 % 4 == 0 and b0 == w0
            if w1 > w0:
                assert b1 == min(n, w1 + w + k - 2)
            covered += list(range(w0, w1))
        assert covered == list(range(nwin))
