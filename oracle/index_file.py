"""Writer (and reader) of the MRQ index file for the CPU oracle.

TEST INFRASTRUCTURE (see ``oracle/mrq.py``).  The GPU library has its own,
independent reader/writer of the same format; the format is the interface the
two share, so that both can search the very same index.

Format (little-endian), version 1:
    char[8] magic "MRQINDEX"; u32 version = 1; u32 n_sections;
    i64 n; i32 D; i32 d; i32 bits; i32 nlist;
    n_sections x { char[4] tag; u32 dtype; u64 count; count elements; zero pad to 8 B }
dtype: 1 = f32, 2 = f64, 3 = i64, 4 = u8.
Sections (required): MU__ f32[D], LAM_ f32[D], W___ f32[D*D] (row-major),
CENT f32[nlist*d], LOFF i64[nlist+1], IDS_ i64[n], CODE u8[n*d] (unsigned level
per dimension), FADD/FRES/FERR f32[n], XD__ f32[n*d], XR__ f32[n*(D-d)], XN2_ f32[n];
optional, B > 1: FRE1/FER1 f32[n], the sign plane's factors (1 bit + refinement);
optional, MR-PQ (Exp-5): PQR_ f32[d*d] the OPQ rotation R (x_d' R is quantized),
PQC_ f32[M*K*(d/M)] the codebooks (subspace-major), PQK_ u8[n*M] the codes (list-major).
Vector arrays are in list-major order (list j holds rows LOFF[j]..LOFF[j+1]-1).
"""
from __future__ import annotations

import struct
import numpy as np

MAGIC = b"MRQINDEX"
VERSION = 1
_DT = {1: np.float32, 2: np.float64, 3: np.int64, 4: np.uint8}
_DT_CODE = {np.dtype(np.float32): 1, np.dtype(np.float64): 2, np.dtype(np.int64): 3,
            np.dtype(np.uint8): 4}


def _sections(idx):
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32).ravel()
    return [
        (b"MU__", f32(idx.mu)), (b"LAM_", f32(idx.lam)), (b"W___", f32(idx.W)),
        (b"CENT", f32(idx.centroids)),
        (b"LOFF", np.ascontiguousarray(idx.list_offsets, dtype=np.int64)),
        (b"IDS_", np.ascontiguousarray(idx.ids, dtype=np.int64)),
        (b"CODE", np.ascontiguousarray(idx.u, dtype=np.uint8).ravel()),
        (b"FADD", f32(idx.f_add)), (b"FRES", f32(idx.f_rescale)), (b"FERR", f32(idx.f_err)),
        (b"XD__", f32(idx.xd)), (b"XR__", f32(idx.xr)), (b"XN2_", f32(idx.xnorm2)),
    ] + ([(b"FRE1", f32(idx.f_rescale1)), (b"FER1", f32(idx.f_err1))]
         if getattr(idx, "f_rescale1", None) is not None else [])


def write_index(idx, path: str, pq=None) -> None:
    """``pq``: optional (R, C, codes) of ``mrq.opq_train`` on idx.xd, written as the
    PQR_ / PQC_ / PQK_ sections."""
    secs = _sections(idx)
    if pq is not None:
        R, C, codes = pq
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32).ravel()
        secs += [(b"PQR_", f32(R)), (b"PQC_", f32(C)),
                 (b"PQK_", np.ascontiguousarray(codes, dtype=np.uint8).ravel())]
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<II", VERSION, len(secs)))
        f.write(struct.pack("<qiiii", idx.n, idx.D, idx.d, idx.bits, idx.nlist))
        for tag, arr in secs:
            f.write(tag)
            f.write(struct.pack("<IQ", _DT_CODE[arr.dtype], arr.size))
            b = arr.tobytes()
            f.write(b)
            pad = (-len(b)) % 8
            if pad:
                f.write(b"\0" * pad)


def read_index(path: str) -> dict:
    """Raw sections of an index file written by ``write_index`` (oracle round trip)."""
    out = {}
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError("not an MRQ index file")
        version, nsec = struct.unpack("<II", f.read(8))
        if version != VERSION:
            raise ValueError("unsupported version")
        n, D, d, bits, nlist = struct.unpack("<qiiii", f.read(24))
        out["header"] = dict(n=n, D=D, d=d, bits=bits, nlist=nlist)
        for _ in range(nsec):
            tag = f.read(4).decode()
            dt, cnt = struct.unpack("<IQ", f.read(12))
            a = np.frombuffer(f.read(cnt * np.dtype(_DT[dt]).itemsize), dtype=_DT[dt])
            pad = (-a.nbytes) % 8
            if pad:
                f.read(pad)
            out[tag] = a
    return out
