"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Parity levels:
* same index: the oracle writes its index file, the GPU library loads it, both
  search it.  Answers must be identical (ids) for every query whose oracle
  decision margin (see ``oracle.mrq.search_contract``) is above float32
  rounding; distances within 2e-5 relative.  Other queries must return valid
  answers (true distances, sorted, almost the same set).
* per candidate: ``mrq_estimate`` on the oracle's projected query against the
  oracle's stage-1 values (Eq. 4 estimate and bounds within 1e-5 relative to the
  distance scale; integer code dot products bit-exact).
* build: GPU mrq_build against oracle build_index on the same draws (PCA,
  rotation, centroids, list membership, codes, factors).
"""
import os

import numpy as np
import pytest

import datagen
from oracle import index_file
from oracle import mrq as omrq

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402

from parity_helpers import DIST_RTOL, STRICT, check_answers  # noqa: E402


def _setup(tmp_path_factory, name, **over):
    w = datagen.workload("small", **over)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=8)
    path = str(tmp_path_factory.mktemp(name) / "index.mrq")
    index_file.write_index(oidx, path)
    return dict(w=w, base=base, queries=queries, G=G, init=init, oidx=oidx,
                stored=oidx.as_stored(), path=path, gidx=mrq.mrq_load(path))


@pytest.fixture(scope="module")
def small(tmp_path_factory):
    return _setup(tmp_path_factory, "small")


@pytest.fixture(scope="module")
def multibit(tmp_path_factory):
    # 4 bits per dimension on d = 64 of D = 128, ragged list sizes
    return _setup(tmp_path_factory, "mb", d=64, bits=4, nlist=50, n=15_000, n_query=120)


@pytest.fixture(scope="module")
def fullrank(tmp_path_factory):
    # d = D: the tail vanishes, MRQ reduces to IVF-RaBitQ
    return _setup(tmp_path_factory, "fr", D=64, d=64, n=8000, n_comp=32, nlist=40, n_query=80)


def _check_answers(S, ids, dists, ref, k, min_strict=0.9, label=""):
    return check_answers(S["base"], S["queries"], np.asarray(ids), np.asarray(dists), ref, k,
                         min_strict=min_strict, label=label)


@pytest.mark.parametrize("qbits", [0, 4])
@pytest.mark.parametrize("mode", [mrq.MODE_MRQ_PLUS, mrq.MODE_MRQ])
def test_same_index_search(small, qbits, mode):
    S = small
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    opts = mrq.mrq_search_opts(mode=mode, query_bits=qbits)
    ids, dists = mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, opts)
    ref = omrq.search_contract(S["stored"], S["queries"], w.k, w.nprobe, mode=mode, qbits=qbits)
    n = _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, w.k, min_strict=0.95,
                       label=f"small mode={mode} qbits={qbits}")
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
    strict = ref.margin > STRICT
    # survivor counts agree up to float32 decisions on irrelevant candidates
    assert np.abs(st["n_s1"] - ref.n_s1)[strict].max() <= max(3, 0.01 * ref.n_s1.max())
    assert np.abs(st["n_exact"] - ref.n_s2)[strict].max() <= max(3, 0.01 * ref.n_s2.max())


@pytest.mark.parametrize("fixture", ["multibit", "fullrank"])
@pytest.mark.parametrize("qbits", [0, 6])
def test_same_index_search_variants(request, fixture, qbits):
    S = request.getfixturevalue(fixture)
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = mrq.mrq_search(S["gidx"], q, w.k, 6, mrq.mrq_search_opts(query_bits=qbits))
    ref = omrq.search_contract(S["stored"], S["queries"], w.k, 6, qbits=qbits)
    _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, w.k)


@pytest.mark.parametrize("k", [1, 32, 100, 200])
def test_k_range(small, k):
    S = small
    q = S["queries"][:40]
    ids, dists = mrq.mrq_search(S["gidx"], q, k, 4)
    ref = omrq.search_contract(S["stored"], q, k, 4)
    strict = ref.margin > STRICT
    np.testing.assert_array_equal(ids[strict], ref.ids[strict])
    np.testing.assert_allclose(dists[strict], ref.dists[strict], rtol=DIST_RTOL, atol=1e-6)


def test_fewer_candidates_than_k_pads(small):
    S = small
    loff = S["stored"].list_offsets
    smallest = int(np.argmin(np.diff(loff)))
    size = int(loff[smallest + 1] - loff[smallest])
    # a query sitting on the smallest list's centroid probes that list first
    qp = np.zeros((1, S["w"].D))
    qp[0, :S["w"].d] = S["stored"].centroids[smallest]
    q = (qp @ S["stored"].W + S["stored"].mu).astype(np.float32)     # W is orthogonal
    k = size + 5
    ids, dists = mrq.mrq_search(S["gidx"], q, k, 1, mrq.mrq_search_opts(eps0=1e9, m=1e9))
    assert np.all(ids[0, size:] == -1) and np.all(np.isinf(dists[0, size:]))
    assert np.all(ids[0, :size] >= 0)


def test_estimate_per_candidate(small, multibit):
    for S in (small, multibit):
        st = S["stored"]
        qd, qr, qr2, sigma, qp2 = omrq.project_queries(st, S["queries"][:6])
        for i in range(6):
            qp32 = np.concatenate([qd[i], qr[i]]).astype(np.float32)
            qd64, qr64 = qp32[:st.d].astype(np.float64), qp32[st.d:].astype(np.float64)
            s64 = float(np.sqrt(np.sum(qr64 ** 2 * st.lam[st.d:])))
            lists, g = omrq.probe(st, qd64, 3)
            for j in lists:
                j = int(j)
                for qbits in (0, 4):
                    got = mrq.mrq_estimate(S["gidx"], qp32, j, mrq.mrq_search_opts(query_bits=qbits))
                    ref = omrq.estimate_list(st, j, qd64, float(g[j]), float(np.sum(qr64 ** 2)),
                                             s64, 1.9, 4.0, qbits)
                    scale = np.maximum(np.abs(ref["dis"]), ref["scale"])
                    assert np.max(np.abs(got["dis"] - ref["dis"]) / scale) < 1e-5
                    assert np.max(np.abs(got["lb"] - ref["lb"]) / scale) < 1e-5
                    assert np.max(np.abs(got["ub"] - ref["ub"]) / scale) < 1e-5
                    if qbits:
                        # integer code dot products are bit-exact where qbar is decisive
                        qprime = (qd64 - st.centroids[j]) / np.sqrt(g[j])
                        q32 = qprime.astype(np.float32)
                        lo, hi = q32.min(), q32.max()
                        t = (q32 - lo) / np.float32((hi - lo) / np.float32(15))
                        if np.min(np.abs(t - np.floor(t) - 0.5)) > 1e-3:
                            np.testing.assert_array_equal(got["int_dot"], ref["int_dot"])


def test_projection(small):
    S = small
    st = S["stored"]
    got = mrq.mrq_project(S["gidx"], S["queries"])
    qd, qr, *_ = omrq.project_queries(st, S["queries"])
    ref = np.concatenate([qd, qr], axis=1)
    scale = np.linalg.norm(S["queries"] - st.mu, axis=1)[:, None]
    assert np.max(np.abs(got - ref) / scale) < 2e-6


def test_batch_invariance_and_host_device(small):
    S = small
    w = S["w"]
    Q = S["queries"]
    ids_all, d_all = mrq.mrq_search(S["gidx"], Q, w.k, w.nprobe)       # host buffers
    qd = torch.from_numpy(Q).cuda()
    ids_dev, d_dev = mrq.mrq_search(S["gidx"], qd, w.k, w.nprobe)      # device buffers
    np.testing.assert_array_equal(ids_all, ids_dev.cpu().numpy())
    np.testing.assert_array_equal(d_all, d_dev.cpu().numpy())
    for a, b in ((0, 1), (1, 8), (8, 71), (71, 200)):
        ids_b, d_b = mrq.mrq_search(S["gidx"], Q[a:b], w.k, w.nprobe)
        np.testing.assert_array_equal(ids_b, ids_all[a:b])
        np.testing.assert_array_equal(d_b, d_all[a:b])


def test_file_round_trip_is_byte_identical(small, tmp_path):
    S = small
    out = str(tmp_path / "again.mrq")
    mrq.mrq_save(S["gidx"], out)
    with open(S["path"], "rb") as f1, open(out, "rb") as f2:
        assert f1.read() == f2.read()


def test_build_matches_oracle(tmp_path):
    w = datagen.workload("small", n=12_000, nlist=40, n_query=50)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 77)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 78)
    for iters in (0, 2):
        oi = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=iters)
        gi = mrq.mrq_build(base, w.d, w.bits, w.nlist,
                           mrq.mrq_build_opts(kmeans_iters=iters, init_ids=init, rotation_gauss=G))
        ex = lambda f: mrq.mrq_index_export(gi, f)
        np.testing.assert_allclose(ex("LAM_"), oi.lam, rtol=1e-5, atol=1e-7 * oi.lam[0])
        np.testing.assert_allclose(ex("MU__"), oi.mu, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(ex("W___"), oi.W, atol=2e-5)
        tol_c = 1e-4 * np.abs(oi.centroids).max()
        np.testing.assert_allclose(ex("CENT"), oi.centroids, atol=tol_c)
        # list membership: identical except points that are (near-)equidistant
        gl, gids = ex("LOFF"), ex("IDS_")
        g_assign = np.empty(w.n, dtype=np.int64)
        o_assign = np.empty(w.n, dtype=np.int64)
        for j in range(w.nlist):
            g_assign[gids[gl[j]:gl[j + 1]]] = j
            o_assign[oi.ids[oi.list_offsets[j]:oi.list_offsets[j + 1]]] = j
        diff = np.nonzero(g_assign != o_assign)[0]
        assert diff.size <= max(2, w.n // 2000)
        # codes and factors for vectors assigned alike
        gpos = np.empty(w.n, dtype=np.int64); gpos[gids] = np.arange(w.n)
        opos = np.empty(w.n, dtype=np.int64); opos[oi.ids] = np.arange(w.n)
        same = np.setdiff1d(np.arange(w.n), diff)
        gc, oc = ex("CODE")[gpos[same]], oi.u[opos[same]]
        c = oi.centroids[o_assign[same]]
        o = (oi.xd[opos[same]] - c) / oi.resid_norm[opos[same]][:, None]
        bad = gc != oc
        assert np.all(np.abs(o[bad]) < 1e-5), "a code bit differs where the sign is decisive"
        ok = ~bad.any(axis=1)
        for f, ref, tol in (("FADD", oi.f_add, 1e-5), ("FRES", oi.f_rescale, 1e-4),
                            ("FERR", oi.f_err, 1e-4), ("XN2_", oi.xnorm2, 1e-5)):
            np.testing.assert_allclose(ex(f)[gpos[same]][ok], ref[opos[same]][ok], rtol=tol,
                                       atol=tol * np.abs(ref).max() * 1e-2)


def test_build_multibit_codes(tmp_path):
    w = datagen.workload("small", n=6000, d=64, bits=3, nlist=24, n_query=10)
    base, _ = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 5)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 6)
    oi = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=0)
    gi = mrq.mrq_build(base, w.d, w.bits, w.nlist,
                       mrq.mrq_build_opts(kmeans_iters=0, init_ids=init, rotation_gauss=G))
    gids = mrq.mrq_index_export(gi, "IDS_")
    if not np.array_equal(gids, oi.ids):
        pytest.skip("a near-equidistant point changed lists")
    gc = mrq.mrq_index_export(gi, "CODE")
    o = (oi.xd - oi.centroids[np.repeat(np.arange(w.nlist), np.diff(oi.list_offsets))]) \
        / oi.resid_norm[:, None]
    t = (2 ** w.bits - 1) / np.abs(o).max(axis=1, keepdims=True)
    y = np.abs(o) * t
    near = (np.abs(o) < 1e-5) | (np.abs(y / 2 - np.round(y / 2)) < 1e-4)
    assert np.all((gc == oi.u) | near)
    assert (gc == oi.u).mean() > 0.999


def test_end_to_end_recall_and_exact_limit():
    w = datagen.workload("small")
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, w.d, w.bits, w.nlist, mrq.mrq_build_opts(seed=11))
    truth, tdist = omrq.exact_knn(base, queries, w.k)
    ids, _ = mrq.mrq_search(gi, queries, w.k, w.nprobe)
    assert omrq.recall_at_k(ids, truth) >= 0.95
    # all lists, bounds that never prune: brute-force k-NN
    ids, dists = mrq.mrq_search(gi, queries, w.k, w.nlist, mrq.mrq_search_opts(eps0=1e9, m=1e9))
    gap = np.diff(tdist, axis=1).min(axis=1) / tdist[:, -1]
    strict = gap > 1e-5
    np.testing.assert_array_equal(ids[strict], truth[strict])
    np.testing.assert_allclose(dists, tdist, rtol=1e-4, atol=1e-5)


def test_empty_lists(tmp_path):
    # initial centroids far from the data leave lists empty
    w = datagen.workload("small", n=3000, nlist=16, n_query=20)
    base, queries = datagen.base_and_queries(w)
    far = np.tile(base.mean(axis=0) + 1e3, (16, 1)).astype(np.float32)
    far[:8] = base[:8]
    gi = mrq.mrq_build(base, w.d, w.bits, 16, mrq.mrq_build_opts(kmeans_iters=0, init_centroids=far))
    sizes = np.diff(mrq.mrq_index_export(gi, "LOFF"))
    assert (sizes == 0).sum() >= 1
    ids, dists = mrq.mrq_search(gi, queries, 5, 16, mrq.mrq_search_opts(eps0=1e9, m=1e9))
    truth, _ = omrq.exact_knn(base, queries, 5)
    assert omrq.recall_at_k(ids, truth) > 0.99


def test_zipf_lists_chunked_scan(tmp_path):
    # rank-size Zipf(1.1) list sizes: the largest lists exceed one scan work item
    # (4096 candidates), so the scan splits them into chunks
    w = datagen.workload("small", n=40_000, nlist=32, n_query=60)
    base, centres, sizes = datagen.zipf_clustered(w, w.n, w.nlist, s=1.1)
    queries = datagen.sample(datagen.make_mixture(w), w.n_query, w.seed("queries"))
    G = datagen.rotation_gaussian(w.d, 9)
    oi = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_centroids=centres, kmeans_iters=0)
    assert np.diff(oi.list_offsets).max() > 2 * 4096
    p = str(tmp_path / "zipf.mrq")
    index_file.write_index(oi, p)
    gi = mrq.mrq_load(p)
    st = oi.as_stored()
    for qbits in (0, 4):
        ids, dists = mrq.mrq_search(gi, queries, w.k, 4, mrq.mrq_search_opts(query_bits=qbits))
        ref = omrq.search_contract(st, queries, w.k, 4, qbits=qbits)
        S = dict(base=base, queries=queries)
        _check_answers(S, ids, dists, ref, w.k)
        stats = mrq.mrq_last_search_stats(gi, w.n_query)
        np.testing.assert_array_equal(stats["n_cand"], ref.n_cand)


@pytest.mark.parametrize("fixture", ["small", "multibit"])
def test_batched_form_equals_per_pair_scan(request, fixture):
    # the list-major batched scan scores every candidate with the same arithmetic
    # and the thresholds are order-independent, so answers are bit-identical
    S = request.getfixturevalue(fixture)
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    for npb in (1, 6, w.nlist):
        a = mrq.mrq_search(S["gidx"], q, w.k, npb, mrq.mrq_search_opts(query_bits=4))
        sa = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
        b = mrq.mrq_search(S["gidx"], q, w.k, npb, mrq.mrq_search_opts(query_bits=4, batched=1))
        sb = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
        np.testing.assert_array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
        np.testing.assert_array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())
        np.testing.assert_array_equal(sa["n_cand"], sb["n_cand"])
        np.testing.assert_array_equal(sa["n_s1"], sb["n_s1"])
    ref = omrq.search_contract(S["stored"], S["queries"], w.k, 6, qbits=4)
    ids, dists = mrq.mrq_search(S["gidx"], q, w.k, 6, mrq.mrq_search_opts(query_bits=4, batched=1))
    _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, w.k)


def test_graph_captured_again_after_scratch_grows(small):
    # a captured graph holds the scratch addresses it was captured with: a larger search
    # in between grows (reallocates) the scratch, and the next call with the same
    # arguments captures again instead of replaying addresses that were freed
    S = small
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    ids = torch.empty((q.shape[0], w.k), dtype=torch.int64, device="cuda")
    dists = torch.empty((q.shape[0], w.k), dtype=torch.float32, device="cuda")
    o = mrq.mrq_search_opts(query_bits=4, graph=1)
    ref_i, ref_d = mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, mrq.mrq_search_opts(query_bits=4))
    mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, o, out=(ids, dists))   # run, capture
    big = torch.cat([q] * 40)
    bi, _ = mrq.mrq_search(S["gidx"], big, w.k, w.nprobe, mrq.mrq_search_opts(query_bits=4))
    np.testing.assert_array_equal(bi[:len(q)].cpu().numpy(), ref_i.cpu().numpy())
    for _ in range(2):
        ids.fill_(-7)
        mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, o, out=(ids, dists))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
        np.testing.assert_array_equal(dists.cpu().numpy(), ref_d.cpu().numpy())


def test_graph_replay(small):
    # a captured search graph replays the same pipeline: identical answers, and new
    # query values written into the same buffer are picked up by the replay
    S = small
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    ids = torch.empty((q.shape[0], w.k), dtype=torch.int64, device="cuda")
    dists = torch.empty((q.shape[0], w.k), dtype=torch.float32, device="cuda")
    for form in (dict(query_bits=4, batched=1), dict(query_bits=0)):
        ref_i, ref_d = mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, mrq.mrq_search_opts(**form))
        for _ in range(3):
            mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, mrq.mrq_search_opts(graph=1, **form),
                           out=(ids, dists))
            torch.cuda.synchronize()
            np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
            np.testing.assert_array_equal(dists.cpu().numpy(), ref_d.cpu().numpy())
        q2 = q.flip(0).contiguous()
        ref2 = mrq.mrq_search(S["gidx"], q2, w.k, w.nprobe, mrq.mrq_search_opts(**form))
        q.copy_(q2)
        mrq.mrq_search(S["gidx"], q, w.k, w.nprobe, mrq.mrq_search_opts(graph=1, **form),
                       out=(ids, dists))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref2[0].cpu().numpy())
        q.copy_(q2.flip(0))
