"""List-sharded search on the GPU (Section 5, distributed deployment): shards made by
mrq_index_shard from an index the oracle wrote, each searched on the GPU, the
answers merged by mrq_merge_topk on the device, against the oracle's search of the
same shards (restrict_lists) merged; the shard contents against the oracle's; the
device merge against the host merge; and the sampled-PCA build against the oracle.

All shards live on the one GPU here; across GPUs the only difference is the
exchange (torch.distributed all_gather), which the gloo CPU test covers."""
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


@pytest.fixture(scope="module")
def setup(tmp_path_factory):
    w = datagen.workload("small", n=16_000, nlist=48, n_query=120)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    path = str(tmp_path_factory.mktemp("shard") / "index.mrq")
    index_file.write_index(oidx, path)
    return dict(w=w, base=base, queries=queries, st=oidx.as_stored(), gidx=mrq.mrq_load(path))


def _gpu_sharded(S, nshards, k, nprobe, opts):
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = [], []
    for s in range(nshards):
        sh = mrq.mrq_index_shard(S["gidx"], nshards, s)
        i, d = mrq.mrq_search(sh, q, k, nprobe, opts)
        ids.append(i)
        dists.append(d)
    return torch.stack(ids), torch.stack(dists)


@pytest.mark.parametrize("nshards", [2, 3])
def test_shard_contents_match_the_oracle_shards(setup, nshards):
    S = setup
    st = S["st"]
    own = mrq.mrq_shard_plan(np.diff(st.list_offsets), nshards)
    total = 0
    for s in range(nshards):
        sh = mrq.mrq_index_shard(S["gidx"], nshards, s)
        ref = omrq.restrict_lists(st, np.nonzero(own == s)[0])
        info = sh.info()
        assert info.n == ref.n and info.nlist == st.nlist and info.d == st.d
        np.testing.assert_array_equal(mrq.mrq_index_export(sh, "LOFF"), ref.list_offsets)
        np.testing.assert_array_equal(mrq.mrq_index_export(sh, "IDS_"), ref.ids)
        np.testing.assert_array_equal(mrq.mrq_index_export(sh, "CODE"), ref.u)
        np.testing.assert_array_equal(mrq.mrq_index_export(sh, "FADD"), ref.f_add.astype(np.float32))
        np.testing.assert_array_equal(mrq.mrq_index_export(sh, "CENT"), st.centroids.astype(np.float32))
        total += info.n
    assert total == st.n


@pytest.mark.parametrize("nshards", [2, 3])
@pytest.mark.parametrize("form", [dict(query_bits=4), dict(query_bits=0),
                                  dict(query_bits=4, batched=mrq.SCAN_BATCHED)])
def test_sharded_search_against_oracle(setup, nshards, form):
    S = setup
    w, st = S["w"], S["st"]
    k, nprobe = w.k, 6
    ids, dists = _gpu_sharded(S, nshards, k, nprobe, mrq.mrq_search_opts(**form))
    gi, gd = mrq.mrq_merge_topk(ids, dists, k)
    own = mrq.mrq_shard_plan(np.diff(st.list_offsets), nshards)
    parts = [omrq.search_contract(omrq.restrict_lists(st, np.nonzero(own == s)[0]),
                                  S["queries"], k, nprobe, qbits=form["query_bits"])
             for s in range(nshards)]
    mi, md = omrq.merge_answers([(p.ids, p.dists) for p in parts], k)

    class Ref:                                    # the merged answer's decision margin
        pass
    ref = Ref()
    ref.ids, ref.dists = mi, md
    # every shard's own decisions, and the gaps between consecutive merged distances up
    # to rank k + 1 (entries of different shards interleave there)
    _, m1 = omrq.merge_answers([(p.ids, p.dists) for p in parts], k + 1)
    with np.errstate(invalid="ignore"):
        gaps = np.diff(m1, axis=1) / np.maximum(m1[:, 1:], 1e-30)
    gaps = np.where(np.isfinite(gaps), gaps, np.inf)
    ref.margin = np.minimum(np.min(np.stack([p.margin for p in parts]), axis=0),
                            gaps.min(axis=1))
    check_answers(S["base"], S["queries"], gi.cpu().numpy(), gd.cpu().numpy(), ref, k,
                  label=f"sharded x{nshards} {form}")


def test_sharded_without_pruning_equals_whole_index(setup):
    S = setup
    w = S["w"]
    q = torch.from_numpy(S["queries"]).cuda()
    opts = mrq.mrq_search_opts(eps0=1e9, m=1e9, query_bits=4)
    wi, wd = mrq.mrq_search(S["gidx"], q, w.k, 8, opts)
    ids, dists = _gpu_sharded(S, 3, w.k, 8, opts)
    gi, gd = mrq.mrq_merge_topk(ids, dists, w.k)
    np.testing.assert_array_equal(gi.cpu().numpy(), wi.cpu().numpy())
    np.testing.assert_array_equal(gd.cpu().numpy(), wd.cpu().numpy())


def test_device_merge_equals_host_merge(setup):
    S = setup
    ids, dists = _gpu_sharded(S, 3, 32, 6, mrq.mrq_search_opts(query_bits=4))
    di, dd = mrq.mrq_merge_topk(ids, dists, 32)
    hi, hd = mrq.mrq_merge_topk(ids.cpu().numpy(), dists.cpu().numpy(), 32)
    np.testing.assert_array_equal(di.cpu().numpy(), hi)
    np.testing.assert_array_equal(dd.cpu().numpy(), hd)
    # padding: a part with no answer at all
    ids2 = torch.cat([ids, torch.full_like(ids[:1], -1)])
    d2 = torch.cat([dists, torch.full_like(dists[:1], float("inf"))])
    pi, pd = mrq.mrq_merge_topk(ids2, d2, 32)
    np.testing.assert_array_equal(pi.cpu().numpy(), hi)


def test_shard_rejections(setup):
    S = setup
    for ns, s in ((0, 0), (2, 2), (S["w"].nlist + 1, 0)):
        with pytest.raises(mrq.MRQError) as e:
            mrq.mrq_index_shard(S["gidx"], ns, s)
        assert e.value.code == mrq.MRQ_EINVAL


def test_sampled_pca_build_matches_oracle():
    w = datagen.workload("small", n=12_000, nlist=32, n_query=10)
    base, _ = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 41)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 42)
    rows = np.sort(np.random.default_rng(43).choice(w.n, 2000, replace=False))
    oi = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=0,
                          pca_rows=rows)
    gi = mrq.mrq_build(base, w.d, w.bits, w.nlist,
                       mrq.mrq_build_opts(kmeans_iters=0, init_ids=init, rotation_gauss=G,
                                          pca_rows=rows))
    ex = lambda f: mrq.mrq_index_export(gi, f)
    np.testing.assert_allclose(ex("MU__"), oi.mu, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(ex("LAM_"), oi.lam, rtol=1e-5, atol=1e-7 * oi.lam[0])
    np.testing.assert_allclose(ex("W___"), oi.W, atol=2e-5)
    assert gi.info().n == w.n
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_build(base, w.d, w.bits, w.nlist, mrq.mrq_build_opts(pca_rows=[0]))
    assert e.value.code == mrq.MRQ_EINVAL
