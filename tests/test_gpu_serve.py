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


def drain(srv, n_expected, timeout=60.0):
    """Collect answers until n_expected arrived: {id: (keys, positions)} copied out, released."""
    got = {}
    import time
    t0 = time.perf_counter()
    while len(got) < n_expected:
        assert time.perf_counter() - t0 < timeout, f"{len(got)} of {n_expected} answers"
        ids, cnt, lat, hp, pp = srv.collect_raw(256, 1.0)
        for i in range(ids.size):
            h, p = B.Server.views(int(cnt[i]), int(hp[i]), int(pp[i]))
            got[int(ids[i])] = (h.copy(), p.copy())
            assert lat[i] >= 0
        srv.release(ids)
    return got


def test_collect_and_release_match_oracle():
    reqs = requests(80, 11) + [(synth.acgt_uniform_packed(7, seed=3).numpy(), 7)]
    srv = B.Server(15, 10, slots=3, max_requests_per_batch=8, max_bases_per_batch=1 << 20)
    try:
        ids = srv.submit_many(reqs)
        got = drain(srv, len(reqs))
        assert sorted(got) == sorted(ids)
        for rid, (seq, n) in zip(ids, reqs):
            rh, rp = oracle.minimizers(seq, n, 15, 10)
            h, p = got[rid]
            assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp)
        with pytest.raises(B.SwsError, match="INVALID"):
            srv.release([ids[0]])  # already released
    finally:
        srv.close()


def test_hbm_budget_holds_a_request_until_the_first_retires():
    n = 300_000
    seqs = [synth.acgt_uniform_packed(n, seed=900 + i).numpy() for i in range(2)]
    one = n // 4 + 24 * n + 64  # device bytes the server reserves for a request of n bases
    for budget, want_batches in ((0, 1), (one + 1, 2)):
        srv = B.Server(15, 10, slots=2, max_requests_per_batch=8, max_bases_per_batch=1 << 20,
                       hbm_budget_bytes=budget)
        try:
            ids = srv.submit_many([(s, n) for s in seqs])  # queued together, in one call
            for rid, s in zip(ids, seqs):
                assert srv.wait(rid, 60.0)
                h, p, _ = srv.result(rid)
                rh, rp = oracle.minimizers(s, n, 15, 10)
                assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp)
            assert srv.stats()["batches"] == want_batches, budget
        finally:
            srv.close()


def test_megabase_requests_match_oracle():
    lens = [1_000_000, 999_999, 1_000_003 - 3, 150, 250_000]
    reqs = [(synth.acgt_uniform_packed(L, seed=70 + i).numpy(), L) for i, L in enumerate(lens)]
    srv = B.Server(15, 10, slots=2, max_requests_per_batch=4, max_bases_per_batch=1 << 21)
    try:
        ids = srv.submit_many(reqs)
        got = drain(srv, len(reqs))
        for rid, (seq, n) in zip(ids, reqs):
            rh, rp = oracle.minimizers(seq, n, 15, 10)
            h, p = got[rid]
            assert np.array_equal(h.astype(np.uint64), rh) and np.array_equal(p, rp), n
    finally:
        srv.close()


def test_held_answers_hold_back_batches_until_released():
    """With one slot the server has four result blocks; answers kept without release hold them,
    later batches wait, and releasing lets every request finish."""
    reqs = requests(12, 5, lo=1000, hi=5000)
    srv = B.Server(15, 10, slots=1, max_requests_per_batch=1, max_bases_per_batch=1 << 16)
    try:
        ids = srv.submit_many(reqs)
        held = []
        import time
        t0 = time.perf_counter()
        while len(held) < 4 and time.perf_counter() - t0 < 30:
            got = srv.collect_raw(16, 0.5)
            held += list(got[0])
        assert len(held) == 4  # every block is held: nothing more is answered
        assert srv.collect_raw(16, 0.3)[0].size == 0
        srv.release(held)
        rest = drain(srv, len(reqs) - 4)
        assert sorted(list(rest) + [int(i) for i in held]) == sorted(ids)
    finally:
        srv.close()
