"""Row-scaled FP8 projection (MRQ_PREC_FP8): every centred query row and every row of
W is scaled to a largest magnitude of 448 and rounded to e4m3; one tcgen05
kind::f8f6f4 product accumulates in float32 and the epilogue applies both scales.

Against the float64 projection with the index's own W and mu (the oracle's file):
each coordinate's error is within the rounding bound of the two e4m3 operands,
sum_i |q_i - mu_i| |W_ji| * ((1 + 2^-4)^2 - 1), plus the subnormal steps; the mean
error is far below it.  Batch invariance, the no-allocation entry point, a search,
and the D % 16 requirement."""
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

U = 2.0 ** -4                       # unit roundoff of e4m3 (3 mantissa bits)
REL = (1 + U) ** 2 - 1              # one product of two rounded operands


@pytest.fixture(scope="module", params=[(960, 128), (256, 64)], ids=["D960", "D256"])
def idx(request, tmp_path_factory):
    D, d = request.param
    w = datagen.workload("small", D=D, d=d, n=8000, n_comp=64, nlist=32, n_query=600)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 3)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 4)
    oi = omrq.build_index(base, w.d, 1, w.nlist, G, init_idx=init, kmeans_iters=4)
    path = str(tmp_path_factory.mktemp(f"fp8_{D}") / "i.mrq")
    index_file.write_index(oi, path)
    st = oi.as_stored()
    return dict(w=w, base=base, queries=queries, st=st, gi=mrq.mrq_load(path))


def test_projection_within_the_e4m3_bound(idx):
    st, q = idx["st"], idx["queries"]
    W = st.W.astype(np.float64)
    qc = q.astype(np.float64) - st.mu.astype(np.float64)
    ref = qc @ W.T
    got = mrq.mrq_project(idx["gi"], torch.from_numpy(q).cuda(),
                          mrq.mrq_search_opts(precision=mrq.PREC_FP8)).cpu().numpy().astype(np.float64)
    D = W.shape[0]
    absq = np.abs(qc)
    bound = REL * (absq @ np.abs(W).T)
    # subnormal steps of the scaled operands: 2^-10 of each row scale per element
    sq = absq.max(axis=1, keepdims=True) / 448
    sw = np.abs(W).max(axis=1)[None, :] / 448
    bound += 2.0 ** -10 * (sq * np.abs(W).sum(axis=1)[None, :] + sw * absq.sum(axis=1, keepdims=True))
    bound += 1e-5 * np.linalg.norm(qc, axis=1, keepdims=True)   # float32 accumulation
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
    rel = err / np.linalg.norm(qc, axis=1, keepdims=True)
    assert rel.mean() < 0.01 and rel.mean() > 0          # rounded: not the exact product
    assert float((err / bound).max()) > 1e-3             # the bound is not vacuous here
    del D


def test_batch_invariance_and_no_alloc(idx):
    gi, q = idx["gi"], torch.from_numpy(idx["queries"]).cuda()
    o = mrq.mrq_search_opts(precision=mrq.PREC_FP8)
    full = mrq.mrq_project(gi, q, o)
    part = mrq.mrq_project(gi, q[:77].contiguous(), o)
    assert torch.equal(full[:77], part)
    out = torch.full_like(full, float("nan"))
    mrq.mrq_project_noalloc(gi, q, out, o)
    assert torch.equal(out, full)


def test_search_recall_close_to_fp32(idx):
    w, gi = idx["w"], idx["gi"]
    q = torch.from_numpy(idx["queries"]).cuda()
    truth, _ = omrq.exact_knn(idx["base"], idx["queries"], 10)
    r = {}
    for name, prec in (("fp32", mrq.PREC_FP32), ("fp8", mrq.PREC_FP8)):
        ids, d = mrq.mrq_search(gi, q, 10, 8, mrq.mrq_search_opts(precision=prec, query_bits=4))
        r[name] = omrq.recall_at_k(ids.cpu().numpy(), truth)
        assert torch.all(d[:, 1:] >= d[:, :-1])
    assert r["fp8"] >= r["fp32"] - 0.05


def test_fp8_needs_rows_of_16_bytes():
    w = datagen.workload("small", D=104, d=32, n=3000, nlist=8, n_query=8)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, 32, 1, 8, mrq.mrq_build_opts(kmeans_iters=1))
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(gi, queries, 5, 2, mrq.mrq_search_opts(precision=mrq.PREC_FP8))
    assert e.value.code == mrq.MRQ_EINVAL and "16" in str(e.value)
