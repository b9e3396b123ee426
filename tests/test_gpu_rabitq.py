"""d = D: no residual tail (sigma = 0 in Eq. 6, every bound is the quantization bound of
Eq. 5 alone), which is IVF-RaBitQ, the paper's main comparison system expressed in
MRQ's own terms.  The code length then reaches the full dimension (up to
MRQ_MAX_D = 1024 here), beyond the shapes of the specialised scan kernels."""
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


# d = 768 runs the generic scan, d = 960 the scan specialised for 30 code words
@pytest.fixture(scope="module", params=[768, 960], ids=["d768", "d960"])
def full_rank(request, tmp_path_factory):
    D = request.param
    w = datagen.workload("small", D=D, d=D, n=6000, n_comp=48, alpha=1.0, nlist=24,
                         n_query=100)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 31)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 32)
    oidx = omrq.build_index(base, w.d, 1, w.nlist, G, init_idx=init, kmeans_iters=4)
    path = str(tmp_path_factory.mktemp(f"fr{D}") / "index.mrq")
    index_file.write_index(oidx, path)
    return dict(w=w, base=base, queries=queries, oidx=oidx, stored=oidx.as_stored(),
                gidx=mrq.mrq_load(path))


@pytest.mark.parametrize("qbits,mode,prec", [(0, mrq.MODE_MRQ_PLUS, mrq.PREC_FP32),
                                             (4, mrq.MODE_MRQ_PLUS, mrq.PREC_BF16X3),
                                             (4, mrq.MODE_MRQ, mrq.PREC_FP32)],
                         ids=["fp32", "q4-bf16x3", "q4-mrq"])
def test_full_rank_same_index(full_rank, qbits, mode, prec):
    S = full_rank
    assert float(np.max(S["stored"].lam[S["w"].d:], initial=0.0)) == 0.0  # no tail
    q = torch.from_numpy(S["queries"]).cuda()
    opts = mrq.mrq_search_opts(query_bits=qbits, mode=mode, precision=prec)
    ids, dists = mrq.mrq_search(S["gidx"], q, 10, 5, opts)
    ref = omrq.search_contract(S["stored"], S["queries"], 10, 5, mode=mode, qbits=qbits)
    _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, 10)
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
    strict = ref.margin > STRICT
    assert np.abs(st["n_s1"] - ref.n_s1)[strict].max() <= max(3, 0.01 * ref.n_s1.max())


def test_full_rank_960_build_without_pruning_is_brute_force():
    """GPU build at d = D = 960 (the GIST dimension), every list probed and bounds too wide
    to prune: the answer is the exact k-NN of the base."""
    w = datagen.workload("small", D=960, d=960, n=5000, n_comp=40, alpha=1.0, nlist=8,
                         n_query=40)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, 960, 1, 8, mrq.mrq_build_opts(seed=9, kmeans_iters=3))
    info = gi.info()
    assert info.d == 960 and info.D == 960
    ref_ids, ref_d = omrq.exact_knn(base, queries, 10)
    for qbits in (0, 4):
        ids, dists = mrq.mrq_search(gi, queries, 10, 8,
                                    mrq.mrq_search_opts(query_bits=qbits, eps0=1e9, m=1e9))
        np.testing.assert_array_equal(ids, ref_ids)
        np.testing.assert_allclose(dists, ref_d, rtol=1e-4, atol=1e-4)
    # with the default bounds the pruned search still finds the neighbours
    ids, _ = mrq.mrq_search(gi, queries, 10, 8, mrq.mrq_search_opts(query_bits=4))
    assert omrq.recall_at_k(ids, ref_ids) > 0.97


def test_dimension_limit():
    w = datagen.workload("small", D=1056, d=1024, n=1500, n_comp=16, nlist=4, n_query=4)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, 1024, 1, 4, mrq.mrq_build_opts(kmeans_iters=1))
    ids, _ = mrq.mrq_search(gi, queries, 5, 4, mrq.mrq_search_opts(eps0=1e9, m=1e9))
    ref_ids, _ = omrq.exact_knn(base, queries, 5)
    np.testing.assert_array_equal(ids, ref_ids)
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_build(base, 1056, 1, 4, mrq.mrq_build_opts(kmeans_iters=1))
    assert e.value.code == mrq.MRQ_EINVAL
