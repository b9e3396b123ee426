"""The optimistic survivor region: when a query's stage-1 survivors overflow the
region its batch gave it, the scan counts them without writing them, lists the
query, and the query is searched again with the full region after the batch.  The
answers must equal those of a search with the full region, bit for bit, in every
scan form, with graph replay, and for k above 32."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402


@pytest.fixture(scope="module")
def zipf():
    w = datagen.workload("small", n=40_000, nlist=32, n_query=300)
    base, centres, _ = datagen.zipf_clustered(w, w.n, w.nlist, s=1.1)
    queries = datagen.sample(datagen.make_mixture(w), w.n_query, w.seed("queries"))
    gi = mrq.mrq_build(base, w.d, 4, w.nlist,
                       mrq.mrq_build_opts(kmeans_iters=0, init_centroids=centres, seed=3))
    return w, queries, gi


@pytest.mark.parametrize("form", [dict(query_bits=4), dict(query_bits=0),
                                  dict(query_bits=4, batched=mrq.SCAN_BATCHED),
                                  dict(query_bits=4, mode=mrq.MODE_MRQ)])
@pytest.mark.parametrize("k", [10, 50])
def test_small_region_gives_the_same_answers(zipf, form, k):
    w, queries, gi = zipf
    q = torch.from_numpy(queries).cuda()
    ref_i, ref_d = mrq.mrq_search(gi, q, k, 6, mrq.mrq_search_opts(eps0=1.9, m=4.0, **form))
    ref_st = mrq.mrq_last_search_stats(gi, len(queries))
    region = 64
    assert (ref_st["n_s1"] > region).sum() >= 10          # many queries overflow it
    got_i, got_d = mrq.mrq_search(gi, q, k, 6, mrq.mrq_search_opts(eps0=1.9, m=4.0,
                                                                   survivor_region=region, **form))
    np.testing.assert_array_equal(got_i.cpu().numpy(), ref_i.cpu().numpy())
    np.testing.assert_array_equal(got_d.cpu().numpy(), ref_d.cpu().numpy())
    st = mrq.mrq_last_search_stats(gi, len(queries))
    np.testing.assert_array_equal(st["n_cand"], ref_st["n_cand"])
    np.testing.assert_array_equal(st["n_exact"], ref_st["n_exact"])


def test_small_region_with_graph_replay_and_host_buffers(zipf):
    w, queries, gi = zipf
    opts = mrq.mrq_search_opts(query_bits=4, survivor_region=64, graph=1)
    ref_i, ref_d = mrq.mrq_search(gi, queries, 10, 6, mrq.mrq_search_opts(query_bits=4))
    q = torch.from_numpy(queries).cuda()
    ids = torch.empty((len(queries), 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((len(queries), 10), dtype=torch.float32, device="cuda")
    for _ in range(3):                                       # run, capture, replay
        mrq.mrq_search(gi, q, 10, 6, opts, out=(ids, dists))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_i)
        np.testing.assert_array_equal(dists.cpu().numpy(), ref_d)
    hi, hd = mrq.mrq_search(gi, queries, 10, 6, mrq.mrq_search_opts(query_bits=4,
                                                                      survivor_region=64))
    np.testing.assert_array_equal(hi, ref_i)
    np.testing.assert_array_equal(hd, ref_d)


def test_negative_region_is_rejected(zipf):
    w, queries, gi = zipf
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(gi, queries[:4], 10, 6, mrq.mrq_search_opts(survivor_region=-1))
    assert e.value.code == mrq.MRQ_EINVAL


@pytest.mark.parametrize("k", [10, 50])
def test_wide_finalize_equals_per_warp_finalize(zipf, k):
    # a batch of few queries with a large region takes the wide finalize (tau_A / tau_B on a
    # CTA per query, gathers split over CTAs); the same queries inside a batch of more than
    # 8192 take the per-warp kernels: the answers and counts are bitwise the same
    w, queries, gi = zipf
    q = torch.from_numpy(queries).cuda()
    o = mrq.mrq_search_opts(eps0=1.9, m=4.0, query_bits=4)
    small_i, small_d = mrq.mrq_search(gi, q, k, 6, o)
    small_st = mrq.mrq_last_search_stats(gi, len(queries))
    reps = 8200 // len(queries) + 1
    big = torch.cat([q] * reps)
    big_i, big_d = mrq.mrq_search(gi, big, k, 6, o)
    big_st = mrq.mrq_last_search_stats(gi, big.shape[0])
    n = len(queries)
    np.testing.assert_array_equal(big_i[:n].cpu().numpy(), small_i.cpu().numpy())
    np.testing.assert_array_equal(big_d[:n].cpu().numpy(), small_d.cpu().numpy())
    for key in ("n_cand", "n_s1", "n_exact"):
        np.testing.assert_array_equal(big_st[key][:n], small_st[key])
