"""mrq_project_noalloc, the projection entry point that allocates no device
memory, against mrq_project on the same index and device queries: two calls
in a row, every precision, the largest batch its static scratch holds, and the
requests it must reject.  It uses the same kernels and tile shapes as
mrq_project, so the outputs are expected to agree to float32 rounding."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2411_06158_gb300 as mrq  # noqa: E402

MAX_BYTES = 8388608          # MRQ_PROJECT_NOALLOC_MAX_BYTES in include/mrq.h
TOL = 1e-6                   # max |noalloc - mrq_project| / |q - mu| per row


@pytest.fixture(scope="module", params=[(128, 64), (960, 128)], ids=["D128", "D960"])
def index(request):
    D, d = request.param
    w = datagen.workload("small", D=D, d=d, n=6000, nlist=16, n_comp=32, n_query=2200)
    base, queries = datagen.base_and_queries(w)
    gi = mrq.mrq_build(base, d, 1, 16, mrq.mrq_build_opts(seed=5, kmeans_iters=4))
    mu = torch.from_numpy(base.astype(np.float64).mean(axis=0).astype(np.float32)).cuda()
    yield D, gi, torch.from_numpy(np.ascontiguousarray(queries, dtype=np.float32)).cuda(), mu
    del gi


def _rel_err(got, ref, q, mu):
    scale = torch.linalg.norm(q - mu, dim=1, keepdim=True).clamp_min(1e-30)
    return float(((got - ref).abs() / scale).max())


@pytest.mark.parametrize("prec", [mrq.PREC_FP32, mrq.PREC_BF16, mrq.PREC_BF16X3, mrq.PREC_FP8],
                         ids=["fp32", "bf16", "bf16x3", "fp8"])
def test_two_calls_match_mrq_project(index, prec):
    D, gi, queries, mu = index
    q = queries[:333].contiguous()                       # ragged: not a multiple of 128 rows
    opts = mrq.mrq_search_opts(precision=prec)
    ref = mrq.mrq_project(gi, q, opts)
    torch.cuda.synchronize()
    outs = [torch.full((q.shape[0], D), float("nan"), device="cuda") for _ in range(2)]
    for out in outs:                                     # two calls in a row
        mrq.mrq_project_noalloc(gi, q, out, opts)
    for out in outs:
        assert torch.isfinite(out).all()
        assert _rel_err(out, ref, q, mu) <= TOL


def _scratch_bytes(prec, nq, D):
    """Scratch one call needs (include/mrq.h): 2 or 4 bytes per element of the bf16
    operand; at FP8 one byte per element rounded up to 256, plus 4 bytes per row scale."""
    if prec == mrq.PREC_FP8:
        return (nq * D + 255) // 256 * 256 + 4 * nq
    return nq * D * (2 if prec == mrq.PREC_BF16 else 4)


def _largest_batch(prec, D):
    lo, hi = 1, MAX_BYTES                      # scratch need grows with nq
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if _scratch_bytes(prec, mid, D) <= MAX_BYTES:
            lo = mid
        else:
            hi = mid - 1
    return lo


def test_fp8_bound_stated_in_the_header():
    assert _largest_batch(mrq.PREC_FP8, 128) == 63550
    assert _largest_batch(mrq.PREC_BF16, 128) * 128 == 4194304
    assert _largest_batch(mrq.PREC_BF16X3, 128) * 128 == 2097152


@pytest.mark.parametrize("prec", [mrq.PREC_BF16, mrq.PREC_BF16X3, mrq.PREC_FP8],
                         ids=["bf16", "bf16x3", "fp8"])
def test_largest_batch_and_rejection(index, prec):
    D, gi, queries, mu = index
    nmax = _largest_batch(prec, D)
    assert _scratch_bytes(prec, nmax + 1, D) > MAX_BYTES
    opts = mrq.mrq_search_opts(precision=prec)
    reps = (nmax + 1 + queries.shape[0] - 1) // queries.shape[0]
    big = queries.repeat(reps, 1)[: nmax + 1].contiguous()
    q = big[:nmax]
    ref = mrq.mrq_project(gi, q, opts)
    out = torch.empty((nmax, D), device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        mrq.mrq_project_noalloc(gi, q, out, opts)
        assert _rel_err(out, ref, q, mu) <= TOL
    # one row more than the static scratch holds: rejected before any launch
    out2 = torch.full((nmax + 1, D), 7.0, device="cuda")
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_project_noalloc(gi, big, out2, opts)
    assert e.value.code == mrq.MRQ_EINVAL
    assert "split the batch" in str(e.value)
    assert bool((out2 == 7.0).all())
    # the scratch is still usable after the rejection
    mrq.mrq_project_noalloc(gi, q, out, opts)
    assert _rel_err(out, ref, q, mu) <= TOL


def test_rejects_host_memory_and_bad_sizes(index):
    D, gi, queries, mu = index
    host_q = queries[:4].cpu().numpy()
    out = torch.empty((4, D), device="cuda")
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_project_noalloc(gi, host_q, out)
    assert e.value.code == mrq.MRQ_EINVAL and "device memory" in str(e.value)
    with pytest.raises(mrq.MRQError) as e:
        mrq.mrq_project_noalloc(gi, queries[:0], out)
    assert e.value.code == mrq.MRQ_EINVAL


def test_device_memory_unchanged_across_calls(index):
    D, gi, queries, mu = index
    q = queries[:512].contiguous()
    outs = {p: torch.empty((512, D), device="cuda")
            for p in (mrq.PREC_FP32, mrq.PREC_BF16, mrq.PREC_BF16X3, mrq.PREC_FP8)}
    for p, out in outs.items():                          # set-up calls
        mrq.mrq_project_noalloc(gi, q, out, mrq.mrq_search_opts(precision=p))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for p, out in outs.items():
            mrq.mrq_project_noalloc(gi, q, out, mrq.mrq_search_opts(precision=p))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
