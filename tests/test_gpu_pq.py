"""MR-PQ on the GPU (Appendix A.2, Exp-5) against the oracle.

* same index: the oracle trains the OPQ (opq_train on x_d') and writes it with its
  index file; the GPU library loads both and searches in MRQ_MODE_PQ; answers against
  search_mrpq (fixed rerank range) on the float32-stored index and OPQ;
* training: mrq_pq_train from the same initial rows and iteration counts against
  opq_train (rotation, codebooks, codes), plus the properties any OPQ must have (R
  orthogonal, every code the nearest centroid of its sub-row under R);
* the OPQ survives save / load and travels with a shard.
"""
import numpy as np
import pytest

import datagen
from oracle import index_file
from oracle import mrq as omrq
from parity_helpers import check_answers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402

M_SUB, K_CB = 32, 16      # d = 64: subspaces of 2 coordinates, 4-bit codes


@pytest.fixture(scope="module")
def pqset(tmp_path_factory):
    w = datagen.workload("small", n=12_000, d=64, nlist=32, n_query=120)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    st = oidx.as_stored()
    pq_init = datagen.kmeans_init_indices(w.n, K_CB, 77)
    R, C, codes = omrq.opq_train(st.xd, M=M_SUB, K=K_CB, init_idx=pq_init, opq_iters=3,
                                 km_iters=4)
    path = str(tmp_path_factory.mktemp("pq") / "index.mrq")
    index_file.write_index(oidx, path, pq=(R, C, codes))
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return dict(w=w, base=base, queries=queries, st=st, pq=(f32(R), f32(C), codes),
                pq_raw=(R, C, codes), pq_init=pq_init, path=path, gidx=mrq.mrq_load(path))


def test_loaded_opq_is_the_oracles(pqset):
    S = pqset
    g = S["gidx"]
    info = g.info()
    assert (info.pq_M, info.pq_K) == (M_SUB, K_CB)
    np.testing.assert_array_equal(mrq.mrq_index_export(g, "PQK_"), S["pq"][2])
    np.testing.assert_array_equal(mrq.mrq_index_export(g, "PQR_"), S["pq"][0].astype(np.float32))


@pytest.mark.parametrize("rerank,k", [(500, 10), (100, 10), (40, 32)])
def test_same_index_search_against_oracle(pqset, rerank, k):
    S = pqset
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = mrq.mrq_search(S["gidx"], q, k, 6, mrq.mrq_search_opts(mode=mrq.MODE_PQ,
                                                                         rerank=rerank))
    ref = omrq.search_mrpq(S["st"], S["queries"], k, 6, S["pq"], rerank=rerank)
    check_answers(S["base"], S["queries"], ids.cpu().numpy(), dists.cpu().numpy(), ref, k,
                  label=f"MR-PQ R={rerank} k={k}")
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
    np.testing.assert_array_equal(st["n_exact"], ref.n_s2)


def test_full_rerank_is_brute_force_over_probed_lists(pqset):
    S = pqset
    w = S["w"]
    ids, _ = mrq.mrq_search(S["gidx"], S["queries"], w.k, w.nlist,
                            mrq.mrq_search_opts(mode=mrq.MODE_PQ, rerank=65536))
    truth, _ = omrq.exact_knn(S["base"], S["queries"], w.k)
    assert omrq.recall_at_k(ids, truth) > 0.999


def test_gpu_training_against_oracle(pqset, tmp_path):
    S = pqset
    g = mrq.mrq_load(S["path"])
    mrq.mrq_pq_train(g, M_SUB, K_CB, opq_iters=3, km_iters=4, init_rows=S["pq_init"])
    R = mrq.mrq_index_export(g, "PQR_").astype(np.float64)
    C = mrq.mrq_index_export(g, "PQC_").astype(np.float64)
    codes = mrq.mrq_index_export(g, "PQK_")
    Ro, Co, co = S["pq_raw"]
    np.testing.assert_allclose(R @ R.T, np.eye(R.shape[0]), atol=2e-5)
    # float32 rows against float64: the same optimum up to a few near-tied assignments
    assert np.mean(codes == co) > 0.995
    np.testing.assert_allclose(R, Ro, atol=2e-3)
    np.testing.assert_allclose(C, Co, atol=2e-3 * np.abs(Co).max())
    # every code is the nearest centroid of its sub-row under the GPU's own R
    Xr = S["st"].xd @ R
    ds = Xr.shape[1] // M_SUB
    for m in range(M_SUB):
        sub = Xr[:, m * ds:(m + 1) * ds]
        dist = np.sum((sub[:, None, :] - C[m][None, :, :]) ** 2, axis=2)
        best = dist.min(axis=1)
        got = dist[np.arange(len(sub)), codes[:, m]]
        assert np.all(got <= best + 1e-4 * np.maximum(best, 1e-6) + 1e-6)
    # distortion of the GPU training against the oracle's
    dec = lambda Cb, cd: omrq.pq_decode(Cb, cd.astype(np.int64))
    e_gpu = np.sum((Xr - dec(C, codes)) ** 2)
    e_ora = np.sum((S["st"].xd @ Ro - dec(Co, co)) ** 2)
    assert abs(e_gpu - e_ora) <= 1e-3 * e_ora
    # a search with the GPU-trained OPQ: the fixed rerank range keeps recall high
    truth, _ = omrq.exact_knn(S["base"], S["queries"], 10)
    ids, _ = mrq.mrq_search(g, S["queries"], 10, 8, mrq.mrq_search_opts(mode=mrq.MODE_PQ))
    assert omrq.recall_at_k(ids, truth) > 0.95
    # save / load keeps the OPQ and the answers
    p = str(tmp_path / "pq.mrq")
    mrq.mrq_save(g, p)
    g2 = mrq.mrq_load(p)
    ids2, _ = mrq.mrq_search(g2, S["queries"], 10, 8, mrq.mrq_search_opts(mode=mrq.MODE_PQ))
    np.testing.assert_array_equal(ids2, ids)


def test_opq_travels_with_a_shard(pqset):
    S = pqset
    st = S["st"]
    own = mrq.mrq_shard_plan(np.diff(st.list_offsets), 2)
    sh = mrq.mrq_index_shard(S["gidx"], 2, 1)
    ref = omrq.restrict_lists(st, np.nonzero(own == 1)[0])
    pos = np.concatenate([np.arange(st.list_offsets[j], st.list_offsets[j + 1])
                          for j in range(st.nlist) if own[j] == 1])
    np.testing.assert_array_equal(mrq.mrq_index_export(sh, "PQK_"), S["pq"][2][pos])
    assert sh.info().n == ref.n


def test_rejections(pqset):
    S = pqset
    w = S["w"]
    plain = mrq.mrq_build(S["base"], w.d, 1, w.nlist, mrq.mrq_build_opts(kmeans_iters=2))
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(plain, S["queries"][:4], 10, 4, mrq.mrq_search_opts(mode=mrq.MODE_PQ))
    assert e.value.code == mrq.MRQ_EINVAL
    for M, K in ((3, 16), (32, 1), (32, 257), (64, 128)):
        with pytest.raises(mrq.MRQError) as e:
            mrq.mrq_pq_train(plain, M, K)
        assert e.value.code == mrq.MRQ_EINVAL
