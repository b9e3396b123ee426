"""The C ABI library loads, exports every entry point that include/mrq.h
declares, and rejects bad arguments and malformed files before touching a GPU."""
import ctypes as C
import os
import re
import struct

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrq.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2411_06158_gb300 as m
    return m


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mrq_build" in names and "mrq_search" in names
    for n in names:
        assert hasattr(lib._lib, n), f"{n} declared in mrq.h but not exported"
    assert set(names) == set(lib.EXPORTS)


def test_defaults(lib):
    o = lib.SearchOpts()
    lib._lib.mrq_search_opts_default(C.byref(o))
    assert o.eps0 == pytest.approx(1.9) and o.m == pytest.approx(4.0)
    assert o.mode == lib.MODE_MRQ_PLUS and o.precision == lib.PREC_FP32
    b = lib.BuildOpts()
    lib._lib.mrq_build_opts_default(C.byref(b))
    assert b.kmeans_iters == 20 and b.seed == 1


@pytest.mark.parametrize("D,d,bits,nlist,msg", [
    (128, 48, 1, 8, "d must be"),        # d not a multiple of 32
    (128, 256, 1, 8, "d must be"),       # d > D
    (128, 32, 0, 8, "bits"),
    (128, 32, 9, 8, "bits"),
    (128, 32, 1, 0, "nlist"),
    (128, 32, 1, 5000, "nlist"),         # nlist > n
    (16, 32, 1, 8, "D must be"),
])
def test_build_rejects_bad_arguments(lib, D, d, bits, nlist, msg):
    base = np.zeros((1000, max(D, 1)), dtype=np.float32)
    h = C.c_void_p()
    rc = lib._lib.mrq_build(base.ctypes.data, 1000, D, d, bits, nlist, None, C.byref(h))
    assert rc == lib.MRQ_EINVAL
    assert msg in lib.mrq_last_error()
    assert h.value is None


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib._lib.mrq_build(None, 10, 64, 32, 1, 2, None, C.byref(h)) == lib.MRQ_EINVAL
    assert lib._lib.mrq_search(None, None, 1, 1, 1, None, None, None) == lib.MRQ_EINVAL
    lib._lib.mrq_free(None)  # no-op


def test_load_rejects_malformed_files(lib, tmp_path):
    h = C.c_void_p()
    assert lib._lib.mrq_load(str(tmp_path / "missing").encode(), C.byref(h)) == lib.MRQ_EIO
    p = tmp_path / "bad"
    p.write_bytes(b"NOTANINDEXFILE" + b"\0" * 64)
    assert lib._lib.mrq_load(str(p).encode(), C.byref(h)) == lib.MRQ_EFORMAT
    p.write_bytes(b"MRQINDEX" + struct.pack("<II", 2, 0))
    assert lib._lib.mrq_load(str(p).encode(), C.byref(h)) == lib.MRQ_EFORMAT
    assert "version" in lib.mrq_last_error()
    p.write_bytes(b"MRQINDEX" + struct.pack("<II", 1, 0) + struct.pack("<qiiii", 10, 64, 48, 1, 2))
    assert lib._lib.mrq_load(str(p).encode(), C.byref(h)) == lib.MRQ_EFORMAT
    p.write_bytes(b"MRQINDEX" + struct.pack("<II", 1, 0))
    assert lib._lib.mrq_load(str(p).encode(), C.byref(h)) == lib.MRQ_EFORMAT
    assert "truncated" in lib.mrq_last_error()


def test_build_script_targets_sm103a():
    import sys
    sys.path.insert(0, os.path.join(ROOT, "paper_2411_06158_gb300"))
    import build_lib
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


STRUCTS = {  # C typedef -> ctypes mirror in the binding
    "mrq_build_opts": "BuildOpts", "mrq_search_opts": "SearchOpts",
    "mrq_index_info_t": "IndexInfo", "mrq_tune_result_t": "TuneResult",
    "mrq_server_opts": "ServerOpts", "mrq_server_stats_t": "ServerStats",
}


def test_struct_layouts_match_the_header(lib, tmp_path):
    """Every option / result struct of include/mrq.h has the size and field offsets of its
    ctypes mirror (a C program built against the header prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mrq.h"', 'int main(void) {']
    for cname, pyname in STRUCTS.items():
        st = getattr(lib, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, pyname in STRUCTS.items():
        st = getattr(lib, pyname)
        assert got[(cname, "size")] == C.sizeof(st), cname
        for f, _ in st._fields_:
            assert got[(cname, f)] == getattr(st, f).offset, f"{cname}.{f}"


def test_new_option_defaults(lib):
    o = lib.SearchOpts()
    lib._lib.mrq_search_opts_default(C.byref(o))
    assert o.refine == 0 and o.rerank == 500 and o.graph == 0 and o.batched == 0
    b = lib.BuildOpts()
    lib._lib.mrq_build_opts_default(C.byref(b))
    assert b.auto_d_variance == pytest.approx(0.8)


def test_build_option_rejections_before_any_gpu_call(lib):
    """Eq. 8's d = 0 cannot take a rotation draw (its size depends on d), its variance
    target must lie in (0, 1], and d may not exceed MRQ_MAX_D = 1024; all rejected by
    argument checks, on a machine without a GPU too."""
    base = np.zeros((2000, 1088), dtype=np.float32)
    h = C.c_void_p()
    o, keep = lib.mrq_build_opts(rotation_gauss=np.zeros((32, 32)))
    rc = lib._lib.mrq_build(base.ctypes.data, 2000, 1088, 0, 1, 8, C.byref(o), C.byref(h))
    assert rc == lib.MRQ_EINVAL and "rotation_gauss" in lib.mrq_last_error()
    for bad in (0.0, -0.5, 1.01):
        o, keep = lib.mrq_build_opts(auto_d_variance=bad)
        rc = lib._lib.mrq_build(base.ctypes.data, 2000, 1088, 0, 1, 8, C.byref(o), C.byref(h))
        assert rc == lib.MRQ_EINVAL and "auto_d_variance" in lib.mrq_last_error()
    rc = lib._lib.mrq_build(base.ctypes.data, 2000, 1088, 1056, 1, 8, None, C.byref(h))
    assert rc == lib.MRQ_EINVAL and "1024" in lib.mrq_last_error()
    assert h.value is None
