"""Tensor-core (tcgen05) paths against the CPU oracle: the bf16 and split hi+lo
bf16 query projection and probe, with ragged query counts and K / N tails.
Expected error (per output, relative to |q - mu|): bf16 rounds each operand to
8 significant bits (~2^-9); hi+lo keeps ~16 bits (~2^-17) before float32
accumulation."""
import numpy as np
import pytest

import datagen
from oracle import mrq as omrq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402
from oracle import index_file  # noqa: E402


def _oracle_index(tmp_path, D, d, n, nlist):
    w = datagen.workload("small", D=D, d=d, n=n, nlist=nlist, n_comp=32, n_query=333)
    base, queries = datagen.base_and_queries(w)
    G = datagen.rotation_gaussian(d, 3)
    init = datagen.kmeans_init_indices(n, nlist, 4)
    oi = omrq.build_index(base, d, 1, nlist, G, init_idx=init, kmeans_iters=3)
    p = str(tmp_path / f"i{D}.mrq")
    index_file.write_index(oi, p)
    return w, base, queries, oi.as_stored(), mrq.mrq_load(p)


@pytest.mark.parametrize("D,d", [(96, 64), (128, 64), (960, 128)])
def test_projection_precisions(tmp_path, D, d):
    w, base, queries, st, gi = _oracle_index(tmp_path, D, d, 4000, 16)
    qd, qr, *_ = omrq.project_queries(st, queries)
    ref = np.concatenate([qd, qr], axis=1)
    scale = np.linalg.norm(queries - st.mu, axis=1)[:, None]
    errs = {}
    for prec in (mrq.PREC_FP32, mrq.PREC_BF16X3, mrq.PREC_BF16):
        got = mrq.mrq_project(gi, queries, mrq.mrq_search_opts(precision=prec))
        errs[prec] = float(np.max(np.abs(got - ref) / scale))
    assert errs[mrq.PREC_FP32] < 2e-6
    assert errs[mrq.PREC_BF16X3] < 5e-5
    assert errs[mrq.PREC_BF16] < 2e-2
    assert errs[mrq.PREC_BF16] > 10 * errs[mrq.PREC_BF16X3]   # the lo half is used


def test_search_precisions_agree(tmp_path):
    w, base, queries, st, gi = _oracle_index(tmp_path, 128, 64, 12000, 48)
    truth, _ = omrq.exact_knn(base, queries, 10)
    res = {}
    for prec in (mrq.PREC_FP32, mrq.PREC_BF16X3, mrq.PREC_BF16):
        ids, dists = mrq.mrq_search(gi, queries, 10, 6, mrq.mrq_search_opts(precision=prec))
        res[prec] = (ids, dists)
    i32, d32 = res[mrq.PREC_FP32]
    i3, d3 = res[mrq.PREC_BF16X3]
    assert np.mean(i3 == i32) > 0.99
    np.testing.assert_allclose(d3[i3 == i32], d32[i3 == i32], rtol=1e-4, atol=1e-5)
    r32 = omrq.recall_at_k(i32, truth)
    assert omrq.recall_at_k(i3, truth) >= r32 - 0.005
    assert omrq.recall_at_k(res[mrq.PREC_BF16][0], truth) >= r32 - 0.05


@pytest.mark.parametrize("graph", [0, 1])
def test_pinned_host_queries_match_device_queries(tmp_path, graph):
    # page-locked host queries are read in place through their device mapping (and the
    # host outputs written by the captured graph); the arithmetic is unchanged, so the
    # answers are bitwise those of the same search on device-resident queries
    w, base, queries, st, gi = _oracle_index(tmp_path, 128, 64, 12000, 48)
    q = np.concatenate([queries] * 16)[:5000].astype(np.float32)
    for prec in (mrq.PREC_BF16, mrq.PREC_BF16X3):
        o = mrq.mrq_search_opts(precision=prec, query_bits=4, graph=graph)
        ref_i, ref_d = mrq.mrq_search(gi, torch.from_numpy(q).cuda(), 10, 6, o)
        qh = torch.from_numpy(q).pin_memory()
        ih = torch.empty((q.shape[0], 10), dtype=torch.int64).pin_memory()
        dh = torch.empty((q.shape[0], 10), dtype=torch.float32).pin_memory()
        for _ in range(2):                                            # capture, then replay
            mrq.mrq_search(gi, qh, 10, 6, o, out=(ih, dh))
            assert torch.equal(ih, ref_i.cpu())
            assert torch.equal(dh, ref_d.cpu())


def test_tensor_core_precision_needs_whole_bf16_rows():
    # bf16 rows of D elements must be 16-byte multiples for the TMA loads: D = 100 is
    # rejected with a clear error before any tensor-core launch; fp32 still works
    w = datagen.workload("small", D=100, d=32, n=3000, nlist=8, n_comp=16, n_query=20)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, 32, 1, 8, mrq.mrq_build_opts(seed=2, kmeans_iters=2))
    ids, _ = mrq.mrq_search(gi, queries, 5, 2, mrq.mrq_search_opts())
    assert ids.shape == (20, 5)
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_search(gi, queries, 5, 2, mrq.mrq_search_opts(precision=mrq.PREC_BF16))
    assert e.value.code == mrq.MRQ_EINVAL and "multiple of 8" in str(e.value)


@pytest.mark.parametrize("D,d,n", [(96, 64, 333), (128, 64, 4097), (960, 128, 1000)])
def test_fused_projection_equals_split_path(tmp_path, D, d, n):
    # 16-byte aligned device queries take the fused projection (float32 rows loaded by
    # TMA, centred and split to bf16 inside the GEMM); the same rows 4 bytes off a
    # 16-byte boundary take the split kernel + GEMM.  One bf16 product per term in the
    # same order: bitwise equal.  The hi+lo form orders its three products per K slice
    # instead of per pass: equal to float32 accumulation rounding.
    w, base, queries, st, gi = _oracle_index(tmp_path, D, d, 4000, 16)
    q = np.concatenate([queries] * (n // len(queries) + 1))[:n].astype(np.float32)
    dev = torch.from_numpy(q).cuda()
    buf = torch.zeros(n * D + 4, dtype=torch.float32, device="cuda")
    buf[1:1 + n * D] = dev.reshape(-1)
    off = buf[1:1 + n * D].view(n, D)
    assert off.data_ptr() % 16 == 4 and dev.data_ptr() % 16 == 0
    scale = np.linalg.norm(q - st.mu, axis=1)[:, None]
    for prec in (mrq.PREC_BF16, mrq.PREC_BF16X3):
        o = mrq.mrq_search_opts(precision=prec)
        a = mrq.mrq_project(gi, dev, o).cpu().numpy()
        b = mrq.mrq_project(gi, off, o).cpu().numpy()
        if prec == mrq.PREC_BF16:
            np.testing.assert_array_equal(a, b)
        else:
            assert float(np.max(np.abs(a - b) / scale)) < 2e-6


def _bf16(x):
    """float32 -> bf16 (round to nearest even), returned as float64"""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("d,nlist,nprobe,nq", [(64, 1000, 3, 1000), (128, 4096, 7, 5000),
                                                (192, 600, 16, 777), (128, 256, 4, 3000)])
def test_fused_probe_selects_the_nearest_lists(prec, d, nlist, nprobe, nq):
    # IVF probing (Algorithm 2) on the tensor cores with the per-row running selection:
    # the lists it probes (seen through the candidate count, a sum of list sizes) are the
    # nprobe smallest g = |q_d'|^2 + |c'|^2 - 2 <bf16 q_d', bf16 c'> recomputed in float64
    # from the GPU's own projected queries and the index's centroids, for every query whose
    # nprobe-th and next g are apart by more than float32 rounding.  Shapes cover one and
    # several query blocks per CTA, ragged list tiles and a zero-filled K slice (d 192).
    w = datagen.workload("small", D=256, d=d, n=max(20 * nlist, 12000), nlist=nlist,
                         n_comp=64, n_query=nq)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, d, 1, nlist, mrq.mrq_build_opts(kmeans_iters=2))
    p = mrq.PREC_BF16 if prec == "bf16" else mrq.PREC_BF16X3
    o = mrq.mrq_search_opts(precision=p, query_bits=4)
    q = torch.from_numpy(queries).cuda()
    mrq.mrq_search(gi, q, 10, nprobe, o)
    n_cand = mrq.mrq_last_search_stats(gi, nq)["n_cand"]
    qd = mrq.mrq_project(gi, q, o).cpu().numpy()[:, :d].astype(np.float64)
    C = mrq.mrq_index_export(gi, "CENT").astype(np.float64)
    sizes = np.diff(mrq.mrq_index_export(gi, "LOFF"))
    qh, ch = _bf16(qd), _bf16(C)
    dot = qh @ ch.T
    if prec == "bf16x3":
        dot += qh @ _bf16(C - ch).T + _bf16(qd - qh) @ ch.T
    g = (qd ** 2).sum(1)[:, None] + (C ** 2).sum(1)[None, :] - 2.0 * dot
    order = np.argsort(g, axis=1, kind="stable")
    gs = np.take_along_axis(g, order, axis=1)
    scale = np.abs(gs[:, :nprobe + 1]).max(axis=1) + 1e-12
    clear = gs[:, nprobe] - gs[:, nprobe - 1] > 1e-5 * scale
    expect = sizes[order[:, :nprobe]].sum(axis=1)
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(n_cand[clear], expect[clear])
