"""CPU oracle of MRQ, written from the paper (arXiv 2411.06158) in plain float64 numpy.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library shares
no code with it.

Parity status of each function is listed in ``oracle/mrq.py``; every function
there is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_pins.py``.
"""
from . import mrq, index_file  # noqa: F401
