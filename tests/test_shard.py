"""List-sharded search (Section 5, distributed deployment) on the CPU: the partition
plan and the host merge of the library, the oracle's shard view, and the one
exchange between two gloo ranks.

The property that makes sharding exact: whenever every bound holds, each shard's
contract answer is the exact top k of its probed candidates, so the merge of the
shards' answers is the exact top k of all probed candidates -- the whole index's
answer (the oracle pins this on its own search)."""
import os
import sys

import numpy as np
import pytest

import datagen
from oracle import mrq as omrq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2411_06158_gb300 as m
    return m


# ------------------------------------------------------------------ partition plan

def test_plan_hand_example(lib):
    # sizes 5 9 1 7 3: 9 -> shard 0, 7 -> 1, 5 -> 1 (7 < 9), 3 -> 0 (9 < 12),
    # 1 -> 0 (12 = 12, lower shard)
    assert lib.mrq_shard_plan([5, 9, 1, 7, 3], 2).tolist() == [1, 0, 0, 1, 0]
    assert lib.mrq_shard_plan([5, 9, 1, 7, 3], 1).tolist() == [0] * 5
    assert sorted(lib.mrq_shard_plan([4, 4, 4], 3).tolist()) == [0, 1, 2]


def test_plan_balance_and_rejections(lib):
    sizes = np.asarray(datagen.zipf_list_sizes(200_000, 512, 1.1, 3), dtype=np.int64)
    for ns in (2, 3, 8):
        own = lib.mrq_shard_plan(sizes, ns)
        load = np.bincount(own, weights=sizes, minlength=ns)
        assert set(own.tolist()) == set(range(ns))
        assert load.max() - load.min() <= sizes.max()
    for bad in ((sizes, 0), (sizes[:2], 3)):
        with pytest.raises(lib.MRQError) as e:
            lib.mrq_shard_plan(*bad)
        assert e.value.code == lib.MRQ_EINVAL


# --------------------------------------------------------------------- host merge

def _sorted_parts(rng, nparts, nq, k, pad_frac=0.2):
    ids = np.full((nparts, nq, k), -1, dtype=np.int64)
    d = np.full((nparts, nq, k), np.inf, dtype=np.float32)
    nxt = 0
    for p in range(nparts):
        for q in range(nq):
            m = int(rng.integers(0, k + 1)) if rng.random() < pad_frac else k
            dv = np.sort(rng.integers(0, 50, m).astype(np.float32) / 8)   # exact ties too
            iv = np.arange(nxt, nxt + m)
            nxt += m
            o = np.lexsort((iv, dv))
            ids[p, q, :m], d[p, q, :m] = iv[o], dv[o]
    return ids, d


@pytest.mark.parametrize("nparts,k", [(1, 5), (2, 10), (3, 1), (7, 32), (40, 16)])
def test_host_merge_against_definition(lib, nparts, k):
    rng = np.random.default_rng(nparts * 100 + k)
    ids, d = _sorted_parts(rng, nparts, 23, k)
    gi, gd = lib.mrq_merge_topk(ids, d, k)
    wi, wd = omrq.merge_answers([(ids[p], d[p]) for p in range(nparts)], k)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gd, wd.astype(np.float32))


def test_merge_rejections(lib):
    ids = np.zeros((65, 1, 1), dtype=np.int64)
    with pytest.raises(lib.MRQError):
        lib.mrq_merge_topk(ids, np.zeros((65, 1, 1), np.float32), 1)
    with pytest.raises(lib.MRQError):
        lib.mrq_merge_topk(ids[:2], np.zeros((2, 1, 1), np.float32), 0)


# ---------------------------------------------- oracle: the shard view, pinned

@pytest.fixture(scope="module")
def sharded(small_workload, small_oracle_index):
    w, base, queries = small_workload
    idx = small_oracle_index
    own = np.arange(idx.nlist) % 3                 # any partition will do for the pins
    shards = [omrq.restrict_lists(idx, np.nonzero(own == s)[0]) for s in range(3)]
    return w, base, queries[:60], idx, shards


def test_shards_partition_the_index(sharded):
    w, base, queries, idx, shards = sharded
    assert sum(s.n for s in shards) == idx.n
    np.testing.assert_array_equal(np.sort(np.concatenate([s.ids for s in shards])),
                                  np.sort(idx.ids))
    for s in shards:
        for j in range(idx.nlist):
            a, b = s.list_slice(j), idx.list_slice(j)
            if a.stop > a.start:
                np.testing.assert_array_equal(s.ids[a], idx.ids[b])
                np.testing.assert_array_equal(s.u[a], idx.u[b])
                np.testing.assert_array_equal(s.f_add[a], idx.f_add[b])


def test_sharded_without_pruning_is_exact_over_probed_lists(sharded):
    w, base, queries, idx, shards = sharded
    k, nprobe = w.k, 6
    parts = [omrq.search_contract(s, queries, k, nprobe, eps0=1e9, m=1e9) for s in shards]
    mi, md = omrq.merge_answers([(p.ids, p.dists) for p in parts], k)
    qd, *_ = omrq.project_queries(idx, queries)
    for i in range(queries.shape[0]):
        lists, _ = omrq.probe(idx, qd[i], nprobe)
        pos = np.concatenate([np.arange(*idx.list_slice(int(j)).indices(idx.n)) for j in lists])
        cand = idx.ids[pos]
        ex = np.sum((base[cand].astype(np.float64) - queries[i]) ** 2, axis=1)
        o = np.lexsort((cand, ex))[:k]
        assert mi[i].tolist() == cand[o].tolist()


def test_sharded_equals_whole_when_bounds_hold(sharded):
    w, base, queries, idx, shards = sharded
    k, nprobe, eps0, m = w.k, 6, 4.0, 12.0
    whole = omrq.search_contract(idx, queries, k, nprobe, eps0=eps0, m=m)
    parts = [omrq.search_contract(s, queries, k, nprobe, eps0=eps0, m=m) for s in shards]
    mi, _ = omrq.merge_answers([(p.ids, p.dists) for p in parts], k)
    qd, qr, qr2, sigma, qp2 = omrq.project_queries(idx, queries)
    checked = 0
    for i in range(queries.shape[0]):
        lists, g = omrq.probe(idx, qd[i], nprobe)
        hold = True
        for j in lists:
            e = omrq.estimate_list(idx, int(j), qd[i], float(g[j]), qr2[i], sigma[i], eps0, m)
            sl = idx.list_slice(int(j))
            ex = np.sum((base[idx.ids[sl]].astype(np.float64) - queries[i]) ** 2, axis=1)
            diso = idx.xnorm2[sl] + qp2[i] - 2.0 * (idx.xd[sl] @ qd[i])
            hold &= bool(np.all((e["lb"] <= ex) & (ex <= e["ub"]))
                         and np.all(np.abs(diso - ex) <= m * sigma[i]))
        if hold:
            checked += 1
            assert mi[i].tolist() == whole.ids[i].tolist()
    assert checked >= 20


# ------------------------------------------------------ sampled PCA (oracle pins)

def test_sampled_pca_over_every_row_is_the_full_pca():
    w = datagen.workload("small", n=3000, n_comp=8, nlist=8, n_query=4)
    base, _ = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 1)
    init = np.arange(8)
    full = omrq.build_index(base, w.d, 1, 8, G, init_idx=init, kmeans_iters=2)
    perm = np.random.default_rng(0).permutation(w.n)
    samp = omrq.build_index(base, w.d, 1, 8, G, init_idx=init, kmeans_iters=2, pca_rows=perm)
    np.testing.assert_allclose(samp.mu, full.mu, rtol=0, atol=1e-12)
    np.testing.assert_allclose(samp.lam, full.lam, rtol=1e-10)
    np.testing.assert_allclose(np.abs(samp.W @ full.W.T), np.eye(w.D), atol=1e-6)


def test_sampled_pca_is_the_pca_of_the_sample():
    w = datagen.workload("small", n=4000, n_comp=8, nlist=8, n_query=4)
    base, _ = datagen.base_and_queries(w)
    rows = np.random.default_rng(2).choice(w.n, 700, replace=False)
    idx = omrq.build_index(base, w.d, 1, 8, datagen.rotation_gaussian(w.d, 1),
                           init_idx=np.arange(8), kmeans_iters=1, pca_rows=rows)
    X = base[rows].astype(np.float64)
    np.testing.assert_allclose(idx.mu, X.mean(axis=0), rtol=0, atol=1e-12)
    sv = np.linalg.svd(X - X.mean(axis=0), compute_uv=False)
    np.testing.assert_allclose(idx.lam, sv ** 2 / len(rows), rtol=1e-9, atol=1e-12)
    # every base row is still indexed, projected with the sample's mean
    assert idx.n == w.n
    xp = (base[idx.ids].astype(np.float64) - idx.mu) @ idx.Pp.T
    np.testing.assert_allclose(np.sum(xp * xp, axis=1), idx.xnorm2, rtol=1e-9)


# -------------------------------------------------- two gloo ranks, one exchange

def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import datagen as dg
    from oracle import mrq as om
    import paper_2411_06158_gb300 as lib
    from paper_2411_06158_gb300 import shard
    w = dg.workload("small", n=8000, n_comp=16, nlist=24, n_query=40)
    base, queries = dg.base_and_queries(w)
    idx = om.build_index(base, w.d, 1, w.nlist, dg.rotation_gaussian(w.d, 5),
                         init_idx=dg.kmeans_init_indices(w.n, w.nlist, 6), kmeans_iters=4)
    own = lib.mrq_shard_plan(np.diff(idx.list_offsets), world)
    mine = om.restrict_lists(idx, np.nonzero(own == rank)[0])
    res = {}
    for name, e0, m in (("exact", 1e9, 1e9), ("bounds", 1.9, 4.0)):
        r = om.search_contract(mine, queries, w.k, 5, eps0=e0, m=m)   # this rank's shard
        ids, d = shard.exchange_and_merge(r.ids, r.dists.astype(np.float32), w.k)
        res[name] = (np.asarray(ids).tolist(), om.search_contract(idx, queries, w.k, 5, eps0=e0,
                                                                  m=m).ids.tolist())
    out[rank] = res
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_and_merge():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = 31500 + (os.getpid() % 2000)
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    # every rank holds the same merged answer
    assert out[0]["exact"][0] == out[1]["exact"][0]
    assert out[0]["bounds"][0] == out[1]["bounds"][0]
    # no pruning: the merge of the shards equals the whole index's answer
    assert out[0]["exact"][0] == out[0]["exact"][1]
    # default bounds: the same answer for nearly every query (bounds hold for most)
    same = np.mean([a == b for a, b in zip(*out[0]["bounds"])])
    assert same >= 0.9
