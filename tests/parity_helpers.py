"""Shared checks of GPU answers against the CPU oracle's contract answers.

Not a test module: the GPU test files import it.  It holds no arithmetic of the
method, only comparisons of answers.
"""
import re

import numpy as np

# A query is compared strictly (identical ids, distances within DIST_RTOL) when
# the oracle's decision margin -- the smallest relative distance of any decision
# that can change its answer from flipping -- exceeds this.  Ties within 1e-6
# are ties; the GPU computes every estimate and distance in float32, whose
# rounding (about 6e-8 per operation, a few operations deep, plus the float32
# projection) stays well below 3e-6 of the distance scale.
STRICT = 3e-6
DIST_RTOL = 2e-5    # float32 distance against the float64 oracle


def check_answers(base, queries, ids, dists, ref, k, strict_margin=STRICT, min_strict=0.95,
                  label=""):
    """Identical ids and close distances for every query whose oracle margin exceeds
    ``strict_margin``; for the others a valid answer: true distances, sorted, and at
    least k - 1 ids in common with the oracle.  Asserts that at least ``min_strict``
    of the queries were compared strictly and prints how many."""
    ids = np.asarray(ids)
    dists = np.asarray(dists)
    strict = ref.margin > strict_margin
    n = int(strict.sum())
    print(f"[parity] {label}: {n} of {strict.size} queries compared strictly "
          f"(margin > {strict_margin:g})")
    assert strict.mean() >= min_strict, f"only {n} of {strict.size} queries decisive"
    np.testing.assert_array_equal(ids[strict], ref.ids[strict])
    np.testing.assert_allclose(dists[strict], ref.dists[strict], rtol=DIST_RTOL, atol=1e-6)
    for qi in np.nonzero(~strict)[0]:
        got = ids[qi][ids[qi] >= 0]
        true = np.sum((base[got].astype(np.float64) - queries[qi]) ** 2, axis=1)
        np.testing.assert_allclose(dists[qi][:got.size], true, rtol=1e-4, atol=1e-5)
        assert np.all(np.diff(dists[qi][:got.size]) >= 0)
        assert len(set(got.tolist()) & set(ref.ids[qi].tolist())) >= k - 1
    return n


def kernels_run(fn):
    """Names of the CUDA kernels ``fn()`` launches (torch profiler, CUPTI), or None
    when the profiler records no device activity on this machine."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    names = set()
    for e in prof.events():
        if str(getattr(e, "device_type", "")).endswith("CUDA"):
            names.add(e.name)
    return names or None


def launched(names, pattern):
    return names is None or any(re.search(pattern, n) for n in names)
