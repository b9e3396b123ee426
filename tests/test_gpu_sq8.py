"""MR-SQ (MRQ_MODE_SQ8, Appendix A.2 Exp-5) on the GPU against the oracle's
``sq8_train`` / ``search_mrsq8``: the SQ8 grid and codes bit-exact (float32 decisions
on both sides), the answers identical wherever the oracle's decision margin is above
float32 rounding, full rerank and full probe equal to brute force, long lists cut into
work items, the rerank range in the graph key, and the rejected requests."""
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
from test_gpu_parity import STRICT, _check_answers  # noqa: E402


def _setup(tmp_path_factory, name, **over):
    w = datagen.workload("small", **over)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=5)
    path = str(tmp_path_factory.mktemp(name) / "index.mrq")
    index_file.write_index(oidx, path)
    st = oidx.as_stored()
    return dict(w=w, base=base, queries=queries, stored=st, sq=omrq.sq8_train(st.xd),
                gidx=mrq.mrq_load(path))


@pytest.fixture(scope="module")
def small(tmp_path_factory):
    return _setup(tmp_path_factory, "sq_small", d=64, n=12_000, nlist=32, n_query=120)


@pytest.fixture(scope="module")
def long_lists(tmp_path_factory):
    # lists of ~6000 vectors: the scan cuts them into 4096-candidate work items
    return _setup(tmp_path_factory, "sq_long", d=96, D=192, n=24_000, nlist=4, n_query=40)


def test_grid_and_codes_bit_exact(small):
    lo, delta, codes = small["sq"]
    g = small["gidx"]
    np.testing.assert_array_equal(mrq.mrq_index_export(g, "SQ8L"), lo)
    np.testing.assert_array_equal(mrq.mrq_index_export(g, "SQ8S"), delta)
    np.testing.assert_array_equal(mrq.mrq_index_export(g, "SQ8C"), codes)


@pytest.mark.parametrize("R,k,prec", [(500, 10, mrq.PREC_FP32), (100, 10, mrq.PREC_BF16X3),
                                      (40, 32, mrq.PREC_FP32)])
def test_mrsq8_matches_oracle(small, R, k, prec):
    S = small
    q = torch.from_numpy(S["queries"]).cuda()
    opts = mrq.mrq_search_opts(mode=mrq.MODE_SQ8, rerank=R, precision=prec)
    ids, dists = mrq.mrq_search(S["gidx"], q, k, 5, opts)
    ref = omrq.search_mrsq8(S["stored"], S["queries"], k, 5, rerank=R, sq=S["sq"])
    n = _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, k)
    assert n >= 0.8 * len(S["queries"])
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
    np.testing.assert_array_equal(st["n_s1"], ref.n_s1)
    np.testing.assert_array_equal(st["n_exact"], np.minimum(R, ref.n_cand))


def test_long_lists_in_work_items(long_lists):
    S = long_lists
    info = S["gidx"].info()
    assert info.max_list > 4096
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = mrq.mrq_search(S["gidx"], q, 10, 2, mrq.mrq_search_opts(mode=mrq.MODE_SQ8))
    ref = omrq.search_mrsq8(S["stored"], S["queries"], 10, 2, rerank=500, sq=S["sq"])
    _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, 10)
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)


def test_full_rerank_full_probe_is_brute_force(small):
    S = small
    w = S["w"]
    Q = S["queries"][:30]
    ref_ids, ref_d = omrq.exact_knn(S["base"], Q, 10)
    ids, dists = mrq.mrq_search(S["gidx"], Q, 10, w.nlist,
                                mrq.mrq_search_opts(mode=mrq.MODE_SQ8, rerank=w.n))
    np.testing.assert_array_equal(ids, ref_ids)
    np.testing.assert_allclose(dists, ref_d, rtol=1e-4, atol=1e-4)


def test_rerank_in_graph_key_and_rejections(small):
    S = small
    q = torch.from_numpy(S["queries"]).cuda()
    ids = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    want = {R: mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(mode=mrq.MODE_SQ8, rerank=R))
            for R in (10, 300)}
    for R in (10, 300, 300, 10):
        mrq.mrq_search(S["gidx"], q, 10, 5,
                       mrq.mrq_search_opts(mode=mrq.MODE_SQ8, rerank=R, graph=1), out=(ids, dists))
        torch.cuda.synchronize()
        assert torch.equal(ids, want[R][0]) and torch.equal(dists, want[R][1])
    for k, R in ((20, 10), (200, 500)):
        with pytest.raises(mrq.MRQError) as e:
            mrq.mrq_search(S["gidx"], q[:4], k, 5, mrq.mrq_search_opts(mode=mrq.MODE_SQ8, rerank=R))
        assert e.value.code == mrq.MRQ_EINVAL
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(S["gidx"], q[:4], 10, 5, mrq.mrq_search_opts(mode=3))
    assert e.value.code == mrq.MRQ_EINVAL


def test_profiled_search(small):
    """Per-stage events also cover the MR-SQ sequence of kernels."""
    S = small
    q = torch.from_numpy(S["queries"]).cuda()
    a = mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(mode=mrq.MODE_SQ8, profile=1))
    ms, launches = mrq.mrq_last_search_profile(S["gidx"])
    assert launches > 0 and all(v >= 0 for v in ms.values())
    b = mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(mode=mrq.MODE_SQ8))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
