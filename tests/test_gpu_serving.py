"""Serving form: continuous batching of requests with mixed k and nprobe.  Every
answer must equal a standalone mrq_search of the same query (the thresholds do
not depend on batch composition), whether it ran alone or in the mix."""
import time

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402


@pytest.fixture(scope="module")
def index():
    w = datagen.workload("small", n=30_000, nlist=96, n_query=600)
    base, queries = datagen.base_and_queries(w)
    return w, queries, mrq.mrq_build(base, w.d, w.bits, w.nlist, mrq.mrq_build_opts(seed=5))


@pytest.mark.parametrize("form", [dict(query_bits=0), dict(query_bits=4, batched=1)])
def test_mixed_requests_match_standalone_search(index, form):
    w, queries, idx = index
    rng = np.random.default_rng(0)
    ks = rng.choice([1, 10, 50, 100], size=len(queries)).astype(np.int32)
    nps = rng.choice([2, 8, 32], size=len(queries)).astype(np.int32)
    opts = mrq.mrq_search_opts(**form)
    srv = mrq.Server(idx, max_batch=64, max_inflight=3, max_wait_us=200, max_k=100, search=opts)
    try:
        tickets = []
        for a in range(0, len(queries), 50):        # arrivals in waves while batches run
            tickets.extend(srv.submit_many(queries[a:a + 50], ks[a:a + 50], nps[a:a + 50]).tolist())
            time.sleep(0.0005)
        lone = srv.submit(queries[7], int(ks[7]), int(nps[7]))   # the same query again, alone
        got, deadline = {}, time.time() + 60
        while len(got) < len(tickets) and time.time() < deadline:
            open_t = [t for t in tickets if t not in got]
            ids, dists, st = srv.poll_many(open_t, 100)
            for i, t in enumerate(open_t):
                assert st[i] in (0, 1)
                if st[i] == 0:
                    got[t] = (ids[i], dists[i])
            time.sleep(0.001)
        # a released ticket is no longer known
        assert srv.poll_many(tickets[:1], 100)[2][0] == mrq.MRQ_EINVAL
        assert len(got) == len(tickets)
        alone = srv.poll(lone, int(ks[7]), wait_ms=10_000)
        assert alone is not None
        stats = srv.stats()
        assert stats["completed"] == len(tickets) + 1 and stats["p99_us"] >= stats["p50_us"] > 0
        assert stats["batches"] >= 9            # nine (k, nprobe) groups at least
    finally:
        srv.stop()
    for i, t in enumerate(tickets):
        k = int(ks[i])
        ref_i, ref_d = mrq.mrq_search(idx, queries[i:i + 1], k, int(nps[i]), opts)
        np.testing.assert_array_equal(got[t][0][:k], ref_i[0])
        np.testing.assert_array_equal(got[t][1][:k], ref_d[0])
    np.testing.assert_array_equal(alone[0], got[tickets[7]][0][:int(ks[7])])


def test_bad_requests_are_rejected(index):
    w, queries, idx = index
    srv = mrq.Server(idx, max_k=16)
    try:
        with pytest.raises(mrq.MRQError):
            srv.submit(queries[0], 17, 4)                       # k above max_k
        with pytest.raises(mrq.MRQError):
            srv.submit(queries[0], 5, w.nlist + 1)              # nprobe above nlist
        with pytest.raises(mrq.MRQError):
            srv.poll(123456, 5)                                  # unknown ticket
    finally:
        srv.stop()


def test_poll_completed_returns_each_ticket_once(index):
    w, queries, idx = index
    srv = mrq.Server(idx, max_batch=128, max_inflight=2, max_wait_us=100, max_k=10)
    try:
        tickets = srv.submit_many(queries[:300], 10, 8)
        seen = {}
        deadline = time.time() + 60
        while len(seen) < 300 and time.time() < deadline:
            tk, ids, dists, st = srv.poll_completed(64, 10)
            for t, i in zip(tk.tolist(), ids):
                assert t not in seen
                seen[t] = i
            time.sleep(0.0005)
        assert sorted(seen) == sorted(tickets.tolist())
        ref, _ = mrq.mrq_search(idx, queries[:300], 10, 8)
        for q, t in enumerate(tickets.tolist()):
            np.testing.assert_array_equal(seen[t], ref[q])
    finally:
        srv.stop()


def test_served_answers_match_the_oracle(tmp_path):
    """Requests with mixed k and nprobe served from an index the oracle wrote, against
    the oracle's contract search of the same index file, query by query."""
    from oracle import index_file
    from oracle import mrq as omrq
    from parity_helpers import check_answers
    w = datagen.workload("small", n=16_000, nlist=48, n_query=160)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    path = str(tmp_path / "served.mrq")
    index_file.write_index(oidx, path)
    gidx = mrq.mrq_load(path)
    st = oidx.as_stored()
    rng = np.random.default_rng(4)
    ks = rng.choice([10, 32], size=len(queries)).astype(np.int32)
    nps = rng.choice([4, 8], size=len(queries)).astype(np.int32)
    srv = mrq.Server(gidx, max_batch=32, max_inflight=3, max_wait_us=200, max_k=32,
                     search=mrq.mrq_search_opts(query_bits=4))
    try:
        tickets = srv.submit_many(queries, ks, nps)
        got, deadline = {}, time.time() + 60
        while len(got) < len(tickets) and time.time() < deadline:
            tk, ids, dists, stt = srv.poll_completed(64, 32)
            for t, i, d in zip(tk.tolist(), ids, dists):
                got[t] = (i, d)
            time.sleep(0.0005)
    finally:
        srv.stop()
    assert len(got) == len(tickets)
    pos = {t: i for i, t in enumerate(tickets.tolist())}
    for k in (10, 32):
        for npb in (4, 8):
            sel = np.nonzero((ks == k) & (nps == npb))[0]
            if sel.size == 0:
                continue
            ref = omrq.search_contract(st, queries[sel], k, npb, qbits=4)
            gi = np.stack([got[int(tickets[i])][0][:k] for i in sel])
            gd = np.stack([got[int(tickets[i])][1][:k] for i in sel])
            # groups of 30-40 queries: one near-tie is already 3 %
            check_answers(base, queries[sel], gi, gd, ref, k, min_strict=0.9,
                          label=f"served k={k} nprobe={npb}")
    assert sorted(pos) == sorted(got)
