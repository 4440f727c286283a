"""The minimizer server (continuous batching): every request's answer equals the oracle's and is
the same whether the request is served alone or in a mix of concurrent requests."""

import threading

import numpy as np
import pytest

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def requests(count, seed, lo=150, hi=200_000):
    lens = synth.loguniform_lengths(count, lo, hi, seed=seed)
    return [(synth.acgt_uniform_packed(int(L), seed=seed * 1000 + i).numpy(), int(L)) for i, L in enumerate(lens)]


def test_served_results_match_oracle_alone_and_in_the_mix():
    reqs = requests(120, 3) + [(synth.acgt_uniform_packed(10, seed=1).numpy(), 10),  # too short: no picks
                               (synth.acgt_uniform_packed(1, seed=2).numpy(), 1)]
    srv = B.Server(15, 10, slots=3, max_requests_per_batch=16, max_bases_per_batch=1 << 20)
    # the mix: all requests submitted at once from two threads
    ids = [None] * len(reqs)

    def submit(part):
        for i in part:
            ids[i] = srv.submit(*reqs[i])

    th = [threading.Thread(target=submit, args=(range(j, len(reqs), 2),)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    mixed = []
    for i, rid in enumerate(ids):
        assert srv.wait(rid, 60.0)
        h, p, lat = srv.result(rid)
        assert lat >= 0
        mixed.append((h, p))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p50_s"] <= st["p99_s"] <= st["max_s"]
    assert st["batches"] > 1
    # alone: one request at a time
    for i, (seq, n) in enumerate(reqs):
        rid = srv.submit(seq, n)
        assert srv.wait(rid, 60.0)
        h, p, _ = srv.result(rid)
        assert np.array_equal(h, mixed[i][0]) and np.array_equal(p, mixed[i][1])
        rh, rp = oracle.minimizers(seq, n, 15, 10)
        assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp), i
    srv.close()


def test_server_limits():
    srv = B.Server(15, 10, slots=1, max_requests_per_batch=4, max_bases_per_batch=4096)
    seq = synth.acgt_uniform_packed(5000).numpy()
    with pytest.raises(B.SwsError, match="CAPACITY"):
        srv.submit(seq, 5000)
    rid = srv.submit(seq, 4096)
    assert srv.wait(rid, 30.0)
    h, p, _ = srv.result(rid)
    rh, rp = oracle.minimizers(seq, 4096, 15, 10)
    assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp)
    srv.close()
    with pytest.raises(B.SwsError, match="UNSUPPORTED"):
        B.Server(19, 10)


def test_submit_many_matches_single_submits():
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 5000, size=200)
    seqs = [synth.acgt_uniform_packed(int(L), seed=500 + i).numpy() for i, L in enumerate(lens)]
    srv = B.Server(15, 10, slots=3, max_requests_per_batch=16, max_bases_per_batch=1 << 16)
    try:
        ids = srv.submit_many([(s, int(L)) for s, L in zip(seqs, lens)])
        assert len(ids) == len(lens) and len(set(ids)) == len(ids)
        for rid, s, L in zip(ids, seqs, lens):
            assert srv.wait(rid, 60.0)
            h, p, _ = srv.result(rid)
            rh, rp = oracle.minimizers(s, int(L), 15, 10)
            assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp)
        with pytest.raises(B.SwsError, match="CAPACITY"):
            srv.submit_many([(seqs[0], int(lens[0])), (np.zeros(1 << 15, np.uint8), 1 << 17)])
    finally:
        srv.close()
