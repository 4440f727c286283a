"""The sharded seed table with its default compute (the CUDA library) on one GPU: a world of one
rank (gloo process group) gives the whole genome's table, equal to the oracle's."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

import oracle
from paper_1811_10074_gb300 import sharded, synth
from gpu_common import random_nblocks, require_gpu

pytestmark = pytest.mark.gpu


def test_single_rank_sharded_table_matches_oracle():
    require_gpu()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        for n, k, w, bb in ((300_001, 15, 10, 16), (200_003, 19, 10, 18)):
            seq = synth.acgt_uniform_packed(n, seed=n).numpy()
            nb = random_nblocks(n, np.random.default_rng(n), 10, 3000)
            sh, sp, off, (bl, bh), before = sharded.sharded_seed_table(seq, n, k, w, bb, nblocks=nb,
                                                                       device=torch.device("cuda", 0))
            mh, mp = oracle.minimizers(seq, n, k, w, nblocks=nb)
            rh, rp, ro = oracle.kmer_table(mh, mp, 2 * k, bb)
            assert (bl, bh, before) == (0, 1 << bb, 0)
            assert np.array_equal(sh, rh) and np.array_equal(sp, rp) and np.array_equal(off, ro)
    finally:
        dist.destroy_process_group()
