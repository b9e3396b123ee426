"""Precision form: the error of every estimated distance against the FP64 oracle.

On an embedding-like sample (unit-norm, anisotropic mixture, spectrum i^-0.8,
D = 768; the shape of the precision-form workload at a size the oracle
finishes in seconds), for d in {64, 128, 256} and each projection precision
(float32 CUDA cores, bf16 and split hi+lo bf16 tensor cores, row-scaled e4m3):

* the query is projected on the GPU at that precision (mrq_project) and the
  stage-1 values of every member of each probed list come from mrq_estimate:
  the Eq. 4 estimate dis', and LB / UB (Eq. 5 plus the Chebyshev term of Eq. 6),
  with a float query and with the 4-bit quantized query;
* the oracle computes the same values in float64 from the raw query on the very
  same index file;
* relative error = |GPU - oracle| / max(|dis'|, f_add + g + |q_r|^2), the
  distance scale of the estimate (the parity tests' measure);
* final distances: the distances mrq_search returns at that precision against
  the exact float64 |x - q|^2 of the same ids, and recall@10 against exact k-NN.

Run with ``-s`` to see the table.  The float32 targets are asserted (estimates
within 1e-5 of the distance scale, final distances within 2e-5); the other
precisions are stated, with sanity bounds only.
"""
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

PRECISIONS = [("fp32", mrq.PREC_FP32), ("bf16", mrq.PREC_BF16), ("bf16x3", mrq.PREC_BF16X3),
              ("fp8", mrq.PREC_FP8)]
NPROBE, K, NQ = 8, 10, 120
EPS0, M = 1.9, 4.0
# sanity ceilings for the reduced precisions (relative to the distance scale)
CEIL = {"fp32": 1e-5, "bf16x3": 1e-4, "bf16": 3e-2, "fp8": 1e-1}


@pytest.fixture(scope="module", params=[64, 128, 256], ids=["d64", "d128", "d256"])
def embed(request, tmp_path_factory):
    d = request.param
    w = datagen.workload("embed", n=40_000, n_comp=128, nlist=64, n_query=NQ, d=d)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    path = str(tmp_path_factory.mktemp("prec") / "index.mrq")
    index_file.write_index(oidx, path)
    truth, _ = omrq.exact_knn(base, queries, K)
    return dict(w=w, base=base, queries=queries, st=oidx.as_stored(), gidx=mrq.mrq_load(path),
                truth=truth)


def _estimate_errors(S, prec, qbits):
    st, gidx, queries = S["st"], S["gidx"], S["queries"]
    qd, qr, qr2, sigma, _ = omrq.project_queries(st, queries)
    qp_gpu = mrq.mrq_project(gidx, queries, mrq.mrq_search_opts(precision=prec))
    e_dis, e_bnd = [], []
    opts = mrq.mrq_search_opts(eps0=EPS0, m=M, query_bits=qbits)
    for i in range(queries.shape[0]):
        lists, g = omrq.probe(st, qd[i], NPROBE)
        for j in lists:
            j = int(j)
            ref = omrq.estimate_list(st, j, qd[i], float(g[j]), qr2[i], sigma[i], EPS0, M, qbits)
            if ref["dis"].size == 0:
                continue
            got = mrq.mrq_estimate(gidx, qp_gpu[i], j, opts)
            scale = np.maximum(np.abs(ref["dis"]), ref["scale"])
            e_dis.append(np.abs(got["dis"] - ref["dis"]) / scale)
            e_bnd.append(np.maximum(np.abs(got["lb"] - ref["lb"]), np.abs(got["ub"] - ref["ub"]))
                         / scale)
    return np.concatenate(e_dis), np.concatenate(e_bnd)


def _final_errors(S, prec):
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = mrq.mrq_search(S["gidx"], q, K, NPROBE,
                                mrq.mrq_search_opts(eps0=EPS0, m=M, precision=prec, query_bits=4))
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy().astype(np.float64)
    ok = ids >= 0
    exact = np.sum((S["base"][np.where(ok, ids, 0)].astype(np.float64)
                    - S["queries"][:, None, :].astype(np.float64)) ** 2, axis=2)
    rel = np.abs(dists - exact)[ok] / np.maximum(exact[ok], 1e-30)
    return rel, omrq.recall_at_k(ids, S["truth"])


@pytest.mark.parametrize("name,prec", PRECISIONS, ids=[p[0] for p in PRECISIONS])
def test_estimated_distance_error_per_precision(embed, name, prec):
    S = embed
    d = S["w"].d
    row, med = {}, {}
    for qbits in (0, 4):
        e_dis, e_bnd = _estimate_errors(S, prec, qbits)
        row[qbits] = (float(e_dis.max()), float(e_dis.mean()), float(e_bnd.max()),
                      float(e_bnd.mean()), e_dis.size)
        med[qbits] = float(np.median(e_dis))
        assert np.all(np.isfinite(e_dis)) and np.all(np.isfinite(e_bnd))
    fin, rec = _final_errors(S, prec)
    print(f"[precision] d={d} {name}: dis' (float query) max {row[0][0]:.2e} mean {row[0][1]:.2e}"
          f" | LB/UB max {row[0][2]:.2e} mean {row[0][3]:.2e}"
          f" | dis' (4-bit query) max {row[4][0]:.2e} mean {row[4][1]:.2e}"
          f" | LB/UB max {row[4][2]:.2e} mean {row[4][3]:.2e}"
          f" | final max {fin.max():.2e} mean {fin.mean():.2e} | recall@10 {rec:.4f}"
          f" | {row[0][4]} estimates")
    ceil = CEIL[name]
    assert row[0][0] <= ceil and row[0][2] <= ceil
    if name == "fp32":
        assert fin.max() <= 2e-5
        # the 4-bit grid may move one level where q' sits at rounding level of a
        # half-step; elsewhere the quantized estimates agree as closely
        assert med[4] <= 1e-6
    assert rec >= 0.8
