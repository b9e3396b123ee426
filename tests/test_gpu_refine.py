"""GPU parity of the 1 bit + refinement stage 1 (refine = 1) against the oracle's
two-level contract (``search_contract(..., refine=True)``): stage 1a scans the sign
plane of every B-bit code with the 1-bit factors, stage 1b computes the full-code
estimate of the stage-1a survivors only.  Same index (the oracle writes it with its
FRE1/FER1 sections, the library loads it), answers identical wherever the oracle's
decision margin is above float32 rounding; plus the build's sign-plane factors, the
file round trip, the graph key and the requests refine must reject."""
import dataclasses

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

# (D, d, bits): sign plane read word by word (d 64, 2 bits), with one 16-byte load
# (d 128, 4 bits), and by the generic scan (3 bits)
SHAPES = {"b2d64": (128, 64, 2), "b4d128": (256, 128, 4), "b3d64": (128, 64, 3)}


def _setup(tmp_path_factory, name):
    D, d, bits = SHAPES[name]
    w = datagen.workload("small", D=D, d=d, bits=bits, nlist=48, n=16_000, n_comp=40,
                         n_query=150)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    path = str(tmp_path_factory.mktemp(name) / "index.mrq")
    index_file.write_index(oidx, path)
    return dict(w=w, base=base, queries=queries, oidx=oidx, stored=oidx.as_stored(),
                path=path, gidx=mrq.mrq_load(path), G=G, init=init)


@pytest.fixture(scope="module", params=list(SHAPES))
def shape(request, tmp_path_factory):
    return _setup(tmp_path_factory, request.param)


@pytest.mark.parametrize("k,qbits,mode", [(10, 4, mrq.MODE_MRQ_PLUS), (10, 3, mrq.MODE_MRQ_PLUS),
                                          (64, 4, mrq.MODE_MRQ_PLUS), (10, 4, mrq.MODE_MRQ)],
                         ids=["k10q4", "k10q3", "k64q4", "k10q4-mrq"])
def test_refine_matches_oracle(shape, k, qbits, mode):
    S = shape
    nprobe = 6
    q = torch.from_numpy(S["queries"]).cuda()
    opts = mrq.mrq_search_opts(mode=mode, query_bits=qbits, refine=1, eps0=1.9, m=4.0)
    ids, dists = mrq.mrq_search(S["gidx"], q, k, nprobe, opts)
    ref = omrq.search_contract(S["stored"], S["queries"], k, nprobe, mode=mode, qbits=qbits,
                               refine=True)
    n = _check_answers(S, ids.cpu().numpy(), dists.cpu().numpy(), ref, k)
    assert n >= 0.8 * len(S["queries"])
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
    strict = ref.margin > STRICT
    assert np.abs(st["n_s1"] - ref.n_s1)[strict].max() <= max(3, 0.01 * ref.n_s1.max())
    assert np.abs(st["n_exact"] - ref.n_s2)[strict].max() <= max(3, 0.01 * ref.n_s2.max())


def test_refine_changes_stage1_not_the_exact_answers(shape):
    """With bounds wide enough to hold, refined and one-stage searches return the same
    exact answers; the refined stage 1 differs (S1 from the two-level thresholds)."""
    S = shape
    q = torch.from_numpy(S["queries"]).cuda()
    kw = dict(query_bits=4, eps0=4.0, m=16.0)
    a_ids, a_d = mrq.mrq_search(S["gidx"], q, 10, 4, mrq.mrq_search_opts(refine=1, **kw))
    b_ids, b_d = mrq.mrq_search(S["gidx"], q, 10, 4, mrq.mrq_search_opts(**kw))
    same = (a_ids == b_ids).all(dim=1).float().mean().item()
    assert same > 0.97
    ref = omrq.search_contract(S["stored"], S["queries"], 10, 4, qbits=4, eps0=4.0, m=16.0,
                               refine=True)
    strict = ref.margin > STRICT
    np.testing.assert_array_equal(a_ids.cpu().numpy()[strict], ref.ids[strict])


def test_build_sign_plane_factors(tmp_path):
    w = datagen.workload("small", n=10_000, d=64, bits=4, nlist=32, n_query=10)
    base, _ = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 21)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 22)
    oi = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=0)
    gi = mrq.mrq_build(base, w.d, w.bits, w.nlist,
                       mrq.mrq_build_opts(kmeans_iters=0, init_ids=init, rotation_gauss=G))
    gids = mrq.mrq_index_export(gi, "IDS_")
    if not np.array_equal(gids, oi.ids):
        pytest.skip("a near-equidistant point changed lists")
    gc = mrq.mrq_index_export(gi, "CODE")
    sign_same = np.all((gc >> 3) == (oi.u >> 3), axis=1)   # identical sign planes
    assert sign_same.mean() > 0.999
    for f, ref in (("FRE1", oi.f_rescale1), ("FER1", oi.f_err1)):
        np.testing.assert_allclose(mrq.mrq_index_export(gi, f)[sign_same], ref[sign_same],
                                   rtol=1e-4, atol=1e-4 * np.abs(ref).max() * 1e-2)
    # a 1-bit index holds no sign-plane factors
    g1 = mrq.mrq_build(base, w.d, 1, w.nlist,
                       mrq.mrq_build_opts(kmeans_iters=0, init_ids=init, rotation_gauss=G))
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_index_export(g1, "FRE1")
    assert e.value.code == mrq.MRQ_EINVAL
    # save / load keeps them, and the loaded index refines identically
    p = str(tmp_path / "g.mrq")
    mrq.mrq_save(gi, p)
    f = index_file.read_index(p)
    np.testing.assert_array_equal(f["FRE1"], mrq.mrq_index_export(gi, "FRE1"))
    np.testing.assert_array_equal(f["FER1"], mrq.mrq_index_export(gi, "FER1"))
    gl = mrq.mrq_load(p)
    _, queries = datagen.base_and_queries(w)
    q = torch.from_numpy(queries).cuda()
    o = mrq.mrq_search_opts(query_bits=4, refine=1)
    a = mrq.mrq_search(gi, q, 10, 5, o)
    b = mrq.mrq_search(gl, q, 10, 5, o)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_one_bit_refine_is_plain(tmp_path_factory):
    S = _setup_one_bit(tmp_path_factory)
    q = torch.from_numpy(S["queries"]).cuda()
    a = mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(query_bits=4, refine=1))
    b = mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(query_bits=4))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _setup_one_bit(tmp_path_factory):
    w = datagen.workload("small", n=6000, nlist=24, n_query=60)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, 3)
    init = datagen.kmeans_init_indices(w.n, w.nlist, 4)
    oidx = omrq.build_index(base, w.d, 1, w.nlist, G, init_idx=init, kmeans_iters=4)
    path = str(tmp_path_factory.mktemp("b1") / "index.mrq")
    index_file.write_index(oidx, path)
    return dict(queries=queries, gidx=mrq.mrq_load(path))


def test_refine_rejections(tmp_path, shape):
    S = shape
    q = torch.from_numpy(S["queries"][:8]).cuda()
    for bad in (dict(query_bits=0, refine=1), dict(query_bits=4, refine=2)):
        with pytest.raises(mrq.MRQError) as e:
            mrq.mrq_search(S["gidx"], q, 10, 4, mrq.mrq_search_opts(**bad))
        assert e.value.code == mrq.MRQ_EINVAL
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(S["gidx"], q, 129, 4, mrq.mrq_search_opts(query_bits=4, refine=1))
    assert e.value.code == mrq.MRQ_EINVAL and "k <= 128" in str(e.value)
    # a file without the optional sections loads, searches, and rejects refine
    old = dataclasses.replace(S["oidx"], f_rescale1=None, f_err1=None)
    p = str(tmp_path / "old.mrq")
    index_file.write_index(old, p)
    gi = mrq.mrq_load(p)
    mrq.mrq_search(gi, q, 10, 4, mrq.mrq_search_opts(query_bits=4))
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(gi, q, 10, 4, mrq.mrq_search_opts(query_bits=4, refine=1))
    assert e.value.code == mrq.MRQ_EINVAL and "FRE1" in str(e.value)


def test_refine_in_graph_key(shape):
    S = shape
    q = torch.from_numpy(S["queries"]).cuda()
    ids = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    want = {}
    for rf in (0, 1):
        want[rf] = mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(query_bits=4, refine=rf))
    for rf in (0, 1, 1, 0, 1):
        mrq.mrq_search(S["gidx"], q, 10, 5, mrq.mrq_search_opts(query_bits=4, refine=rf, graph=1),
                       out=(ids, dists))
        torch.cuda.synchronize()
        assert torch.equal(ids, want[rf][0]) and torch.equal(dists, want[rf][1])
