"""The scan autotuner: every configuration it times returns the same answer (the
threshold contract does not depend on the work decomposition), the choice it
records is what batched=SCAN_AUTO then runs, and that answer equals the per-pair
scan's bitwise.  Lists of about a thousand vectors make the chunk size a real choice."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402


@pytest.fixture(scope="module")
def zipf_index():
    w = datagen.workload("small", D=128, d=64, n=60000, nlist=64, n_comp=64, n_query=3000)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, 64, 1, 64, mrq.mrq_build_opts(seed=3, kmeans_iters=2))
    return gi, queries


@pytest.mark.parametrize("k,nprobe", [(10, 4), (50, 16)])
def test_autotune_consistent_and_used(zipf_index, k, nprobe):
    gi, queries = zipf_index
    q = torch.from_numpy(queries).cuda()
    o_auto = mrq.mrq_search_opts(query_bits=4, precision=mrq.PREC_BF16, batched=mrq.SCAN_AUTO)
    r = mrq.mrq_autotune(gi, q, k, nprobe, o_auto)
    assert r["consistent"] == 1
    assert r["n_tried"] >= 2
    assert r["scan"] in (mrq.SCAN_PAIRS, mrq.SCAN_BATCHED, mrq.SCAN_BATCHED_TC)
    assert r["chunk"] in (1024, 4096, 16384) and 1 <= r["group"] <= 16
    assert 0 < r["ms"] <= r["ms_default"] * 1.25   # timing noise aside, no worse than the rule
    ids_a, d_a = mrq.mrq_search(gi, q, k, nprobe, o_auto)
    o_pair = mrq.mrq_search_opts(query_bits=4, precision=mrq.PREC_BF16, batched=mrq.SCAN_PAIRS)
    ids_p, d_p = mrq.mrq_search(gi, q, k, nprobe, o_pair)
    assert torch.equal(ids_a, ids_p) and torch.equal(d_a, d_p)
    o_b = mrq.mrq_search_opts(query_bits=4, precision=mrq.PREC_BF16, batched=mrq.SCAN_BATCHED)
    ids_b, d_b = mrq.mrq_search(gi, q, k, nprobe, o_b)
    assert torch.equal(ids_b, ids_p) and torch.equal(d_b, d_p)


def test_bad_scan_mode_rejected(zipf_index):
    gi, queries = zipf_index
    o = mrq.mrq_search_opts(batched=4)
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(gi, queries[:4], 10, 4, o)
    assert e.value.code == mrq.MRQ_EINVAL


@pytest.mark.parametrize("d,bits", [(64, 1), (128, 2), (128, 4), (256, 4)])
def test_tensor_core_scan_matches_popcount_scans(d, bits):
    # the tensor-core batched scan computes the integer code dots with a bf16 MMA;
    # they are exact, so the answers (and counters) equal both popcount scans bitwise
    w = datagen.workload("small", D=max(2 * d, 128), d=d, n=30000, nlist=32, n_comp=64,
                         n_query=1500, bits=bits)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, d, bits, 32, mrq.mrq_build_opts(seed=7, kmeans_iters=3))
    q = torch.from_numpy(queries).cuda()
    res = {}
    for mode in (mrq.SCAN_PAIRS, mrq.SCAN_BATCHED, mrq.SCAN_BATCHED_TC):
        o = mrq.mrq_search_opts(query_bits=4, precision=mrq.PREC_BF16, batched=mode)
        ids, dists = mrq.mrq_search(gi, q, 10, 6, o)
        res[mode] = (ids, dists, mrq.mrq_last_search_stats(gi, q.shape[0]))
    for mode in (mrq.SCAN_BATCHED, mrq.SCAN_BATCHED_TC):
        assert torch.equal(res[mode][0], res[mrq.SCAN_PAIRS][0])
        assert torch.equal(res[mode][1], res[mrq.SCAN_PAIRS][1])
        for key in ("n_cand", "n_s1", "n_exact"):
            np.testing.assert_array_equal(res[mode][2][key], res[mrq.SCAN_PAIRS][2][key])
