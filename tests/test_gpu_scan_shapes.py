"""Oracle parity of every compiled scan shape (Eq. 4, Eq. 5, Algorithm 2 stage 1).

The per-pair scan with a 4-bit query is compiled per code shape (bits per
dimension B, d/32 code words per plane) for k <= 32 and for 32 < k <= 128; the
batched scan and the tensor-core batched scan cover d a multiple of 128.  Each
shape here runs on an index the oracle wrote (the GPU library loads the same
file) and its answers are compared with the oracle's contract answers, query by
query.  The GIST-like shape the benchmark runs (D 960, d 128, 1 bit, 4-bit
query) has its own case, for the per-pair scan (k 10 and k 50), the batched
scans and the plain float32 form.
"""
import numpy as np
import pytest

import datagen
from oracle import index_file
from oracle import mrq as omrq
from parity_helpers import check_answers, kernels_run, launched

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402

# (bits, d) of every shape the per-pair quantized scan is specialised for
FIXED_SHAPES = [(1, 32), (1, 64), (1, 128), (1, 256), (2, 64), (2, 128), (2, 256),
                (4, 32), (4, 128), (4, 256)]
NPROBE = 6

_cache = {}


def _index(tmp_path_factory, name, **over):
    key = (name, tuple(sorted(over.items())))
    if key in _cache:
        return _cache[key]
    w = datagen.workload(name, **over)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    oidx = omrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=6)
    path = str(tmp_path_factory.mktemp("shape") / "index.mrq")
    index_file.write_index(oidx, path)
    S = dict(w=w, base=base, queries=queries, stored=oidx.as_stored(), gidx=mrq.mrq_load(path),
             refs={})
    _cache[key] = S
    return S


def _ref(S, k, nprobe, qbits, mode=omrq.MODE_MRQ_PLUS):
    key = (k, nprobe, qbits, mode)
    if key not in S["refs"]:
        S["refs"][key] = omrq.search_contract(S["stored"], S["queries"], k, nprobe, qbits=qbits,
                                              mode=mode)
    return S["refs"][key]


def _search(S, k, nprobe, **opts):
    q = torch.from_numpy(S["queries"]).cuda()
    ids, dists = mrq.mrq_search(S["gidx"], q, k, nprobe, mrq.mrq_search_opts(**opts))
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dists.cpu().numpy()


def _shape_index(tmp_path_factory, bits, d):
    return _index(tmp_path_factory, "small", n=12_000, D=256, d=d, bits=bits, nlist=32,
                  n_comp=32, n_query=150)


@pytest.mark.parametrize("bits,d", FIXED_SHAPES)
@pytest.mark.parametrize("k", [10, 50])
def test_fixed_scan_shape_against_oracle(tmp_path_factory, bits, d, k):
    S = _shape_index(tmp_path_factory, bits, d)
    ref = _ref(S, k, NPROBE, 4)
    km = 0 if k <= 32 else 1
    pat = rf"k_scan_q<{km}, ?{d // 32}, ?{bits}, ?4"
    box = {}
    names = kernels_run(lambda: box.update(r=_search(S, k, NPROBE, query_bits=4)))
    assert launched(names, pat), f"{pat} not among {sorted(names or [])}"
    ids, dists = box["r"]
    check_answers(S["base"], S["queries"], ids, dists, ref, k,
                  label=f"per-pair k_scan_q B={bits} d={d} k={k}")
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)


# the popcount batched scan holds a candidate's code in one lane (at most 16 words of a
# power-of-two count); the tensor-core scan takes d a multiple of 128 and B <= 4
BATCHED_CASES = ([(mrq.SCAN_BATCHED, b, d) for b, d in [(1, 32), (1, 128), (1, 256), (2, 128),
                                                          (4, 128)]]
                 + [(mrq.SCAN_BATCHED_TC, b, d) for b, d in [(1, 128), (1, 256), (2, 128),
                                                               (4, 128), (4, 256)]])


@pytest.mark.parametrize("scan,bits,d", BATCHED_CASES)
def test_batched_scans_against_oracle(tmp_path_factory, scan, bits, d):
    S = _shape_index(tmp_path_factory, bits, d)
    k = 10
    ref = _ref(S, k, NPROBE, 4)
    pat = r"k_scan_tc" if scan == mrq.SCAN_BATCHED_TC else r"k_scan_batched"
    box = {}
    names = kernels_run(lambda: box.update(r=_search(S, k, NPROBE, query_bits=4, batched=scan)))
    assert launched(names, pat), f"{pat} not among {sorted(names or [])}"
    ids, dists = box["r"]
    check_answers(S["base"], S["queries"], ids, dists, ref, k,
                  label=f"{pat} B={bits} d={d}")


@pytest.fixture(scope="module")
def gist_shape(tmp_path_factory):
    # the benchmark's shape (GIST-like D 960, d 128, 1 bit) on 20k vectors
    return _index(tmp_path_factory, "gist", n=20_000, n_comp=64, nlist=64, n_query=150)


@pytest.mark.parametrize("k", [10, 50])
def test_bench_shape_per_pair_scan(gist_shape, k):
    S = gist_shape
    ref = _ref(S, k, NPROBE, 4)
    pat = rf"k_scan_q<{0 if k <= 32 else 1}, ?4, ?1, ?4"
    box = {}
    names = kernels_run(lambda: box.update(r=_search(S, k, NPROBE, query_bits=4)))
    assert launched(names, pat), f"{pat} not among {sorted(names or [])}"
    ids, dists = box["r"]
    check_answers(S["base"], S["queries"], ids, dists, ref, k, label=f"GIST-like d128 k={k}")
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)


@pytest.mark.parametrize("form", [dict(query_bits=4, batched=mrq.SCAN_BATCHED),
                                  dict(query_bits=4, batched=mrq.SCAN_BATCHED_TC),
                                  dict(query_bits=4, mode=mrq.MODE_MRQ),
                                  dict(query_bits=0)])
def test_bench_shape_other_forms(gist_shape, form):
    S = gist_shape
    k = 10
    ref = _ref(S, k, NPROBE, form["query_bits"], form.get("mode", omrq.MODE_MRQ_PLUS))
    ids, dists = _search(S, k, NPROBE, **form)
    check_answers(S["base"], S["queries"], ids, dists, ref, k, label=f"GIST-like d128 {form}")


@pytest.mark.parametrize("nprobe", [33, 40, 64])
def test_probe_selection_above_32_lists(gist_shape, nprobe):
    # nprobe > 32: the distance matrix is written and the CTA selection picks the lists
    # (linear buckets over the row's range, an exact sort of the candidates)
    S = gist_shape
    ref = _ref(S, 10, nprobe, 4)
    ids, dists = _search(S, 10, nprobe, query_bits=4)
    check_answers(S["base"], S["queries"], ids, dists, ref, 10, label=f"GIST-like nprobe={nprobe}")
    st = mrq.mrq_last_search_stats(S["gidx"], len(S["queries"]))
    np.testing.assert_array_equal(st["n_cand"], ref.n_cand)
