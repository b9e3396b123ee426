import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def small_workload():
    """The small plain workload (N=20k, D=128, d=32, 1 bit, 64 lists), seeded."""
    import datagen
    w = datagen.workload("small")
    base, queries = datagen.base_and_queries(w)
    return w, base, queries


@pytest.fixture(scope="session")
def small_oracle_index(small_workload):
    import datagen
    from oracle import mrq
    w, base, _ = small_workload
    G = datagen.rotation_gaussian(w.d, w.seed("method"))
    init = datagen.kmeans_init_indices(w.n, w.nlist, w.seed("method") + 1)
    return mrq.build_index(base, w.d, w.bits, w.nlist, G, init_idx=init, kmeans_iters=10)
