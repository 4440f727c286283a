"""Batched minimizers replayed as one CUDA graph (sws_batch_*) against the per-read oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import require_gpu, to_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def make_batch(rng, nreads, lo, hi, seed):
    lens = rng.integers(lo, hi + 1, size=nreads)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    seq = synth.acgt_uniform_packed(int(offs[-1]), seed=seed)
    return seq, offs


def check_run(bt, seq, offs, k, w, mode="hash"):
    nreads = offs.size - 1
    total = int(offs[-1])
    bt.load(seq.cuda(), torch.from_numpy(offs).cuda())
    bt.run(nreads, total)
    h, p, po = bt.results()
    rh, rp, rpo = oracle.minimizers_batch(seq, offs, k, w, mode)
    assert (po.cpu().numpy().view(np.uint64) == rpo).all()
    assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()
    return h.numel()


@pytest.mark.parametrize("options", ["default", "lookback", "tune"])
def test_batch_graph_replays_any_size(options):
    rng = np.random.default_rng({"default": 1, "lookback": 2, "tune": 3}[options])
    bt = B.Batch(max_reads=3000, max_bases=600_000, k=15, w=10, options=options)
    if options == "tune":  # all three paths timed: staged, look-back, single pass
        assert all(t > 0 for t in bt.tuned_ms) and bt.path in (0, 1, 2)
    assert bt.path == {"default": 2, "lookback": 1}.get(options, bt.path)
    batches = [make_batch(rng, 2000, 100, 250, 11), make_batch(rng, 30, 1000, 20000, 12),
               make_batch(rng, 3000, 0, 30, 13), make_batch(rng, 1, 50, 50, 14), make_batch(rng, 2999, 150, 199, 15)]
    for seq, offs in batches:
        check_run(bt, seq, offs, 15, 10)
    # an empty batch
    bt.run(0, 0)
    h, p, po = bt.results()
    assert h.numel() == 0 and int(po[0]) == 0
    # the same batch again, after others: identical output
    seq, offs = batches[0]
    assert check_run(bt, seq, offs, 15, 10) > 0
    bt.close()


@pytest.mark.parametrize("options", ["default", "lookback"])
def test_batch_wide_keys(options):
    """k = 19 (38-bit hashes): the single pass on 64-bit keys, or the look-back kernel."""
    rng = np.random.default_rng(5)
    bt = B.Batch(max_reads=500, max_bases=200_000, k=19, w=10, options=options)
    assert bt.path == {"default": 2, "lookback": 1}[options]
    for i in range(2):
        seq, offs = make_batch(rng, 400, 60, 400, 20 + i)
        check_run(bt, seq, offs, 19, 10)
    bt.close()


@pytest.mark.parametrize("k,w", [(16, 17), (5, 4)])
def test_batch_single_pass_graph(k, w):
    """The default graph for hashed k-mers with k <= 16 and 4 <= w <= 17 is the single pass, the
    sizes read from the device descriptor at every replay."""
    rng = np.random.default_rng(k + w)
    bt = B.Batch(max_reads=4000, max_bases=400_000, k=k, w=w)
    assert bt.path == 2
    for lo, hi, nreads in ((100, 250, 1500), (0, 3 * (k + w), 4000), (20_000, 90_000, 4), (k + 40, k + 40, 1)):
        seq, offs = make_batch(rng, nreads, lo, hi, int(rng.integers(1 << 30)))
        if offs[-1] <= 400_000:
            check_run(bt, seq, offs, k, w)
    bt.close()


def test_batch_rejects_oversized_runs():
    bt = B.Batch(max_reads=10, max_bases=1000, k=15, w=10)
    with pytest.raises(B.SwsError, match="INVALID"):
        bt.run(11, 100)
    with pytest.raises(B.SwsError, match="INVALID"):
        bt.run(5, 1001)
    bt.close()
