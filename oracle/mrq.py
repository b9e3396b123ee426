"""Plain FP64 CPU oracle of MRQ (projection + quantization AKNN, arXiv 2411.06158).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run anything under ``oracle/``.  The
GPU library never calls it, and it shares no code with the GPU library: the two
meet only at the index file format and at the seeded inputs of ``datagen``.

Everything is float64 unless a step below says otherwise.  Readings of points
the paper leaves open (centering, the multi-bit code, the query quantizer, the
order-independent threshold contract ...) are listed in the docstrings of the
functions that implement them.

Notation (Section 4): x_p = P_p (x - mu) is the PCA-rotated vector, x_d its first
d coordinates, x_r the rest; c is the IVF centroid of x's list; P_r a random
orthogonal d x d matrix.  Everything after the random rotation is stored in the
rotated frame: x_d' = P_r^T x_d, c' = P_r^T c, so that o' = P_r^T (x_d - c)/|x_d - c|
is the vector whose signs RaBitQ keeps (Section 4.2).  The combined projection
W = [P_r^T P_p[:d]; P_p[d:]] maps a centred raw vector straight to [x_d' | x_r].
"""
from __future__ import annotations

import dataclasses
import math
import numpy as np

__all__ = [
    "OracleIndex", "choose_d", "pca_train", "orthogonal_from_gaussian", "kmeans", "encode",
    "build_index", "project_queries", "probe", "quantize_query", "estimate_list",
    "search_contract", "search_literal", "exact_knn", "SearchResult", "sq8_train",
    "sq8_estimate", "search_mrsq8", "opq_train", "pq_decode", "pq_estimate", "search_mrpq",
    "restrict_lists", "merge_answers",
]

MODE_MRQ = 0
MODE_MRQ_PLUS = 1


# --------------------------------------------------------------------------- build

def choose_d(lam, D: int, target: float = 0.8, max_d: int = 1024) -> int:
    """Eq. 8 (Section 5, parameter setting): d = the smallest power of two 2^i >= 128
    whose leading PCA coordinates hold at least `target` of the total variance.

    Reading (the printed formula is garbled): the sums run over the variances
    lam_j = sigma_j^2 (the prose speaks of captured variance), the denominator over all
    D coordinates.  d is a multiple of 32 no larger than D (nor than the library's
    largest quantized dimension): when no power of two below that cap reaches the
    target, d is the cap itself.
    """
    lam = np.maximum(np.asarray(lam, dtype=np.float64)[:D], 0.0)
    total = float(lam.sum())
    cap = min((D // 32) * 32, max_d)
    p = 128
    while p < cap:
        if float(lam[:p].sum()) >= target * total:
            return p
        p *= 2
    return cap


def pca_train(S: np.ndarray):
    """PCA of the base set (Algorithm 1, first two steps; residual variances of Eq. 6).

    Reading: the data is centred by its mean mu before rotation (Eq. 6 assumes
    zero-mean data) and the covariance uses 1/N.  sigma_i^2 of Eq. 6 is the i-th
    eigenvalue lam_i of this covariance.  Eigenvectors are sign-normalised so
    that their entry of largest magnitude is positive (lowest index on ties).

    Returns mu (D), lam (D, descending), Pp (D x D, rows are eigenvectors).
    """
    X = np.asarray(S, dtype=np.float64)
    n = X.shape[0]
    mu = X.mean(axis=0)
    Xc = X - mu
    cov = (Xc.T @ Xc) / n
    w, V = np.linalg.eigh(cov)           # ascending
    order = np.argsort(-w, kind="stable")
    lam = w[order]
    Pp = V[:, order].T.copy()
    for i in range(Pp.shape[0]):
        j = int(np.argmax(np.abs(Pp[i])))
        if Pp[i, j] < 0:
            Pp[i] = -Pp[i]
    return mu, lam, Pp


def orthogonal_from_gaussian(G: np.ndarray) -> np.ndarray:
    """Random orthogonal P_r of Algorithm 1 from a Gaussian draw G: the Q factor of
    G = QR with diag(R) > 0 (unique, Haar-distributed)."""
    Q, R = np.linalg.qr(np.asarray(G, dtype=np.float64))
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def _sqdist(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """All squared distances |x - c|^2 (rows of X against rows of C)."""
    return (np.sum(X * X, axis=1)[:, None] + np.sum(C * C, axis=1)[None, :]
            - 2.0 * (X @ C.T))


def _assign(X: np.ndarray, C: np.ndarray, block: int = 16384) -> np.ndarray:
    out = np.empty(X.shape[0], dtype=np.int64)
    for s in range(0, X.shape[0], block):
        out[s:s + block] = np.argmin(_sqdist(X[s:s + block], C), axis=1)  # first min = lowest id
    return out


def kmeans(X: np.ndarray, init: np.ndarray, iters: int):
    """Lloyd's k-means for the IVF centroids (Algorithm 1, IVF training step).

    Readings: ``iters`` rounds of (assign to nearest centroid, ties to the lower
    id; move each centroid to the mean of its members; an empty list keeps its
    centroid), then a final assignment to the final centroids.
    Returns (centroids, assignment).
    """
    C = np.array(init, dtype=np.float64, copy=True)
    for _ in range(iters):
        a = _assign(X, C)
        cnt = np.bincount(a, minlength=C.shape[0]).astype(np.float64)
        sums = np.zeros_like(C)
        np.add.at(sums, a, X)
        nz = cnt > 0
        C[nz] = sums[nz] / cnt[nz][:, None]
    return C, _assign(X, C)


def encode(o: np.ndarray, bits: int):
    """Quantization code of unit vectors o' (rows), RaBitQ-style (Section 4.2).

    1 bit/dim (the paper's code): u_i = [o'_i > 0]; the code vector is
    v = 2u - 1 (the sign vector), so <v, o'>/|v| is RaBitQ's <x_bar, x>.

    B > 1 bits/dim (reading; the paper fixes only "arbitrary" code lengths):
    v_i is an odd integer in {+-1, +-3, ..., +-(2^B - 1)} with the sign of o'_i and
    magnitude the odd integer nearest to |o'_i| * t, t = (2^B - 1)/max_i |o'_i|;
    the stored unsigned level is u_i = (v_i + 2^B - 1)/2 in [0, 2^B - 1].  The
    level decision is taken in float32 (the GPU kernel's precision).  With B = 1
    this is exactly the sign code.  A zero vector gets u = 0.

    Returns (u uint8 [n x d], v float64 [n x d]).
    """
    o = np.asarray(o, dtype=np.float64)
    top = (1 << bits) - 1
    o32 = o.astype(np.float32)
    pos = o32 > 0
    if bits == 1:
        lev = np.ones_like(o32)
    else:
        a32 = np.abs(o32)
        mx = a32.max(axis=1, keepdims=True)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(mx > 0, np.float32(top) / mx, np.float32(0)).astype(np.float32)
        y = (a32 * t).astype(np.float32)
        lev = (np.float32(2) * np.floor(y * np.float32(0.5)) + np.float32(1)).astype(np.float32)
        lev = np.clip(lev, 1, top)
    v = np.where(pos, lev, -lev).astype(np.float64)
    zero = ~np.any(o32 != 0, axis=1)
    v[zero] = -float(top)
    u = ((v + top) / 2).astype(np.uint8)
    return u, v


@dataclasses.dataclass
class OracleIndex:
    """IVF-MRQ index (Algorithm 1 outputs), arrays in list-major order."""
    D: int
    d: int
    bits: int
    nlist: int
    mu: np.ndarray          # D
    lam: np.ndarray         # D, descending eigenvalues (sigma_i^2 of Eq. 6)
    Pp: np.ndarray          # D x D
    Pr: np.ndarray          # d x d
    W: np.ndarray           # D x D = [Pr^T Pp[:d]; Pp[d:]]
    centroids: np.ndarray   # nlist x d, rotated frame c'
    list_offsets: np.ndarray  # nlist + 1
    ids: np.ndarray         # n, original ids in list-major order
    xd: np.ndarray          # n x d, rotated lead coordinates x_d'
    xr: np.ndarray          # n x (D - d), tail coordinates x_r
    xnorm2: np.ndarray      # n, |x_p|^2
    u: np.ndarray           # n x d uint8 code levels
    v: np.ndarray           # n x d code values (odd integers)
    f_add: np.ndarray       # n, |x_d - c|^2 + |x_r|^2
    f_rescale: np.ndarray   # n, -2 |x_d - c| / <v, o'>
    f_err: np.ndarray       # n, 2 |x_d - c| sqrt((1 - a^2)/a^2)/sqrt(d - 1), a = <v,o'>/|v|
    ip_vo: np.ndarray       # n, <v, o'>
    resid_norm: np.ndarray  # n, |x_d - c|
    # 1-bit factors of the sign plane (B > 1 only; None for B = 1): the factors the
    # sign code v1 = 2*(u >> (B-1)) - 1 -- exactly the 1-bit code of o' -- would have
    f_rescale1: np.ndarray | None = None
    f_err1: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.ids.shape[0])

    def list_slice(self, j: int) -> slice:
        return slice(int(self.list_offsets[j]), int(self.list_offsets[j + 1]))

    def as_stored(self) -> "OracleIndex":
        """The index as the file format stores it: every real array rounded to
        float32 (then held in float64 for arithmetic)."""
        r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
        r1 = lambda a: None if a is None else r(a)
        return dataclasses.replace(
            self, mu=r(self.mu), lam=r(self.lam), W=r(self.W), centroids=r(self.centroids),
            xd=r(self.xd), xr=r(self.xr), xnorm2=r(self.xnorm2), f_add=r(self.f_add),
            f_rescale=r(self.f_rescale), f_err=r(self.f_err),
            f_rescale1=r1(self.f_rescale1), f_err1=r1(self.f_err1))


def factors(resid_norm: np.ndarray, xr2: np.ndarray, v: np.ndarray, o: np.ndarray, d: int):
    """Per-vector constants of Eq. 4 and Eq. 5 (Algorithm 1, precomputation step).

    dis' = f_add + |q_d - c|^2 + |q_r|^2 + f_rescale * |q_d - c| * <v, q'>   (Eq. 4)
    eps_b = eps0 * |q_d - c| * f_err                                      (Eq. 5)
    Eq. 5's D is read as the quantized dimension d.  A vector on its centroid
    (|x_d - c| = 0) gets f_rescale = f_err = 0.
    """
    ip = np.sum(v * o, axis=1)
    vn = np.sqrt(np.sum(v * v, axis=1))
    a = np.where(vn > 0, ip / np.where(vn > 0, vn, 1), 0)
    ok = resid_norm > 0
    safe_ip = np.where(ok, ip, 1.0)
    safe_a = np.where(ok, a, 1.0)
    f_add = resid_norm ** 2 + xr2
    f_rescale = np.where(ok, -2.0 * resid_norm / safe_ip, 0.0)
    f_err = np.where(ok, 2.0 * resid_norm * np.sqrt(np.maximum(1.0 - safe_a ** 2, 0.0) / safe_a ** 2)
                     / math.sqrt(d - 1), 0.0)
    return f_add, f_rescale, f_err, ip


def build_index(S, d: int, bits: int, nlist: int, G: np.ndarray, *,
                init_idx: np.ndarray | None = None, init_centroids: np.ndarray | None = None,
                kmeans_iters: int = 20, pca_rows: np.ndarray | None = None) -> OracleIndex:
    """Algorithm 1: PCA, rotate, split, IVF on x_d, quantize with P_r, precompute.

    ``G`` is the d x d Gaussian draw behind P_r.  The initial centroids are the
    base points ``init_idx`` (projected) or the raw-space points
    ``init_centroids`` (projected); one of the two is required.
    ``pca_rows``: the PCA (mean, covariance, eigenvalues) is taken over these base
    rows only -- the sampled global statistics Section 5 suggests for data spread over
    many machines; every row is still projected, clustered and encoded.
    """
    S = np.asarray(S, dtype=np.float64)
    n, D = S.shape
    if not (0 < d <= D and d % 32 == 0 and 1 <= bits <= 8 and 1 <= nlist <= n and d >= 2):
        raise ValueError("invalid build parameters")
    # PCA matrix and residual variances
    mu, lam, Pp = pca_train(S if pca_rows is None else S[np.asarray(pca_rows)])
    Xp = (S - mu) @ Pp.T                             # x_p = P_p x (centred)
    xd, xr = Xp[:, :d], Xp[:, d:]                    # split
    if init_centroids is not None:
        init = ((np.asarray(init_centroids, dtype=np.float64) - mu) @ Pp.T)[:, :d]
    else:
        init = xd[np.asarray(init_idx)]
    C, assign = kmeans(xd, init, kmeans_iters)        # IVF on the projected vectors
    Pr = orthogonal_from_gaussian(G)
    xd_rot = xd @ Pr                                 # rows: P_r^T x_d
    C_rot = C @ Pr
    resid = xd_rot - C_rot[assign]
    rn = np.sqrt(np.sum(resid * resid, axis=1))
    o = np.where(rn[:, None] > 0, resid / np.where(rn > 0, rn, 1)[:, None], 0.0)
    u, v = encode(o, bits)                           # quantize with P_r
    xr2 = np.sum(xr * xr, axis=1)
    f_add, f_rescale, f_err, ip = factors(rn, xr2, v, o, d)
    fr1 = fe1 = None
    if bits > 1:                                     # factors of the sign plane (refinement)
        v1 = 2.0 * (u >> (bits - 1)).astype(np.float64) - 1.0
        _, fr1, fe1, _ = factors(rn, xr2, v1, o, d)
    order = np.lexsort((np.arange(n), assign))      # list-major, ids ascending inside a list
    counts = np.bincount(assign, minlength=nlist)
    offs = np.zeros(nlist + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    W = np.vstack([Pr.T @ Pp[:d], Pp[d:]])
    xn2 = np.sum(xd_rot * xd_rot, axis=1) + xr2
    return OracleIndex(D=D, d=d, bits=bits, nlist=nlist, mu=mu, lam=lam, Pp=Pp, Pr=Pr, W=W,
                       centroids=C_rot, list_offsets=offs, ids=order.astype(np.int64),
                       xd=xd_rot[order], xr=xr[order], xnorm2=xn2[order], u=u[order], v=v[order],
                       f_add=f_add[order], f_rescale=f_rescale[order], f_err=f_err[order],
                       ip_vo=ip[order], resid_norm=rn[order],
                       f_rescale1=None if fr1 is None else fr1[order],
                       f_err1=None if fe1 is None else fe1[order])


def restrict_lists(idx: OracleIndex, lists) -> OracleIndex:
    """One shard of a list-sharded index (Section 5, distributed deployment): the same
    statistics, rotation and centroids (so it probes the same lists), holding only the
    members of ``lists``; every other list is empty.  Row order inside a list is kept."""
    keep = np.zeros(idx.nlist, dtype=bool)
    keep[np.asarray(lists, dtype=np.int64)] = True
    sizes = np.where(keep, np.diff(idx.list_offsets), 0)
    rows = np.concatenate([np.arange(idx.list_offsets[j], idx.list_offsets[j + 1])
                           for j in range(idx.nlist) if keep[j]] or [np.zeros(0, np.int64)])
    offs = np.zeros(idx.nlist + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    sel = lambda a: None if a is None else a[rows]
    return dataclasses.replace(
        idx, list_offsets=offs, ids=idx.ids[rows], xd=idx.xd[rows], xr=idx.xr[rows],
        xnorm2=idx.xnorm2[rows], u=idx.u[rows], v=idx.v[rows], f_add=idx.f_add[rows],
        f_rescale=idx.f_rescale[rows], f_err=idx.f_err[rows], ip_vo=idx.ip_vo[rows],
        resid_norm=idx.resid_norm[rows], f_rescale1=sel(idx.f_rescale1), f_err1=sel(idx.f_err1))


def merge_answers(parts, k: int):
    """The k smallest (distance, id) of each query over several answers (the shards'),
    padding (id -1) ignored; returns (ids, dists) padded with -1 / +inf."""
    nq = parts[0][0].shape[0]
    ids = np.full((nq, k), -1, dtype=np.int64)
    dists = np.full((nq, k), np.inf)
    for q in range(nq):
        pairs = sorted((float(d_), int(i_)) for pi, pd in parts
                       for i_, d_ in zip(pi[q], pd[q]) if i_ >= 0)[:k]
        for t, (d_, i_) in enumerate(pairs):
            ids[q, t], dists[q, t] = i_, d_
    return ids, dists


# -------------------------------------------------------------------------- search

def project_queries(idx: OracleIndex, Q: np.ndarray):
    """Algorithm 2, query preparation: q_p = P_p (q - mu), split into q_d and q_r,
    and the residual standard deviation of Eq. 6, sigma^2 = sum_{i>d} q_i^2 sigma_i^2.
    Returns (qd' [nq x d] in the rotated frame, qr [nq x (D-d)], qr2, sigma, qp2)."""
    qp = (np.asarray(Q, dtype=np.float64) - idx.mu) @ idx.W.T
    qd, qr = qp[:, :idx.d], qp[:, idx.d:]
    qr2 = np.sum(qr * qr, axis=1)
    sigma = np.sqrt(np.sum(qr * qr * idx.lam[idx.d:][None, :], axis=1))
    qp2 = np.sum(qd * qd, axis=1) + qr2
    return qd, qr, qr2, sigma, qp2


def probe(idx: OracleIndex, qd: np.ndarray, nprobe: int):
    """IVF probing (Algorithm 2): the nprobe centroids nearest to q_d, ascending
    |q_d - c|^2, ties to the lower list id.  Returns (lists, g) of one query,
    plus the full g vector."""
    g = np.sum((idx.centroids - qd[None, :]) ** 2, axis=1)
    order = np.lexsort((np.arange(idx.nlist), g))
    return order[:nprobe], g


def quantize_query(qprime: np.ndarray, qbits: int):
    """Scalar quantization of the normalised, rotated query q' (Algorithm 2's
    "quantize query" step).  Reading: a uniform grid between min and max of q'
    with 2^qbits levels, deterministic round-half-up floor(t + 1/2) taken in
    float32.  Returns (qbar int64, v_l, delta) with q' ~ v_l + delta * qbar."""
    q32 = np.asarray(qprime, dtype=np.float32)
    lo = np.float32(q32.min())
    hi = np.float32(q32.max())
    top = np.float32((1 << qbits) - 1)
    delta = np.float32((hi - lo) / top)
    if delta > 0:
        t = ((q32 - lo) / delta).astype(np.float32)
        qbar = np.floor(t + np.float32(0.5)).astype(np.int64)
        qbar = np.clip(qbar, 0, (1 << qbits) - 1)
    else:
        qbar = np.zeros(q32.shape, dtype=np.int64)
    return qbar, float(lo), float(delta)


def estimate_list(idx: OracleIndex, j: int, qd, g_j, qr2, sigma, eps0, m,
                  qbits: int = 0, sign_plane: bool = False):
    """Stage (1) for every member of list j (Eq. 4 and the bounds of Algorithm 2).

    ip = <v, q'> with q' = (q_d' - c_j')/sqrt(g_j), exactly (qbits = 0) or through
    the quantized query (qbits > 0): with q' ~ v_l + delta*qbar and
    v = 2u - (2^B - 1),
        <v, q'> ~ delta*(2<u,qbar> - (2^B-1) sum(qbar)) + v_l*(2 sum(u) - d(2^B-1)).
    dis' = f_add + g_j + |q_r|^2 + f_rescale * sqrt(g_j) * ip          (Eq. 4)
    eps_b = eps0 * sqrt(g_j) * f_err  (Eq. 5),  eps_r = m * sigma  (Chebyshev, Eq. 6)
    LB = dis' - eps_b - eps_r, UB = dis' + eps_b + eps_r.
    Returns dict with ip, dis, lb, ub (and the integer dot when quantized).

    sign_plane: the first level of the 1-bit + refinement scan of a B > 1 code: the
    same estimate from the sign plane alone (u1 = u >> (B-1), v1 = 2 u1 - 1, the
    1-bit code of o') with its own factors f_rescale1, f_err1.
    """
    sl = idx.list_slice(j)
    sg = math.sqrt(g_j)
    qprime = (qd - idx.centroids[j]) / sg if g_j > 0 else np.zeros(idx.d)
    out = {}
    if sign_plane:
        u = (idx.u[sl] >> (idx.bits - 1)).astype(np.int64)
        top = 1
        vcode = 2.0 * u - 1.0
        fres, ferr = idx.f_rescale1[sl], idx.f_err1[sl]
    else:
        u = idx.u[sl].astype(np.int64)
        top = (1 << idx.bits) - 1
        vcode = idx.v[sl]
        fres, ferr = idx.f_rescale[sl], idx.f_err[sl]
    if qbits > 0:
        qbar, vl, delta = quantize_query(qprime, qbits)
        dot = u @ qbar
        su = u.sum(axis=1)
        ip = delta * (2.0 * dot - top * float(qbar.sum())) + vl * (2.0 * su - idx.d * top)
        out.update(int_dot=dot, qbar=qbar, vl=vl, delta=delta)
    else:
        ip = vcode @ qprime
    dis = idx.f_add[sl] + g_j + qr2 + fres * sg * ip
    eps = eps0 * sg * ferr + m * sigma
    out.update(ip=ip, dis=dis, lb=dis - eps, ub=dis + eps, scale=idx.f_add[sl] + g_j + qr2)
    return out


def _decision_margin(lb, ub, sc, tau, k, rel) -> float:
    """Smallest relative distance of a relevant decision lb_i <= tau from flipping.
    A candidate among the k smallest upper bounds (ub_i <= tau) is kept for sure
    while it stays among them (lb_i <= ub_i <= tau), so its margin is the larger
    of |lb_i - tau| and the gap between the k-th and (k+1)-th upper bounds; this
    covers zero-width bounds (d = D, where lb = ub)."""
    srt = np.sort(ub)
    gap_k = (srt[k] - srt[k - 1]) / max(abs(srt[k]), 1e-30) if srt.size > k else math.inf
    m = np.abs(lb - tau) / sc
    top = ub <= tau
    m = np.where(top, np.maximum(m, gap_k), m)
    return float(np.min(m[rel]))


def _kth(values: np.ndarray, k: int) -> float:
    return float(np.partition(values, k - 1)[k - 1]) if values.size >= k else math.inf


@dataclasses.dataclass
class SearchResult:
    ids: np.ndarray         # nq x k (int64, -1 padded)
    dists: np.ndarray       # nq x k (+inf padded)
    n_cand: np.ndarray      # candidates scanned per query
    n_s1: np.ndarray        # stage-1 survivors
    n_s2: np.ndarray        # stage-2 survivors (= exact distance computations)
    margin: np.ndarray      # per query: smallest relative distance of any decision to its threshold


def search_contract(idx: OracleIndex, Q, k: int, nprobe: int, *, eps0: float = 1.9,
                    m: float = 4.0, mode: int = MODE_MRQ_PLUS, qbits: int = 0,
                    refine: bool = False) -> SearchResult:
    """Algorithm 2 under the order-independent threshold contract.

    The paper's loop prunes against the running k-th exact distance, which
    depends on visit order.  The contract replaces it by order statistics of
    per-candidate quantities (reading, used by the GPU path):
      tau_A = k-th smallest UB1 over all probed candidates,  S1 = {LB1 <= tau_A};
      MRQ+ (stage 2, Eq. 7): dis_o' = |x_p|^2 + |q_p|^2 - 2<x_d, q_d>,
      LB2/UB2 = dis_o' -+ m*sigma, tau_B = min(tau_A, k-th smallest UB2 over S1),
      S2 = {i in S1 : LB2 <= tau_B};  MRQ (no stage 2): S2 = S1.
    The answer is the k smallest exact |x_p - q_p|^2 over S2, ties by id.
    refine (B > 1: 1 bit + refinement): stage 1 runs in two levels, the sign plane
    first (LB1a/UB1a with the 1-bit factors), then the full code on its survivors:
      tau_A' = k-th smallest UB1a,  S1a = {LB1a <= tau_A'},
      tau_A = min(tau_A', k-th smallest UB1b over S1a),  S1 = {i in S1a : LB1b <= tau_A}.
    Whenever every bound holds, the answer equals the exact top-k of the probed
    lists (and so does the paper's sequential loop).

    ``margin`` records, per query, the smallest relative gap of any decision
    that can change the answer: the probed/unprobed centroid boundary, the
    stage-1 test of a candidate that is in the answer, could enter it (exact
    distance within the k-th) or could move tau_B (its UB2 among the k smallest),
    the stage-2 test of an answer-relevant candidate, and consecutive answer
    distances around rank k.  An implementation computing in float32 may
    legitimately answer differently only where this gap is at rounding level.
    """
    qd_all, qr_all, qr2_all, sig_all, qp2_all = project_queries(idx, Q)
    nq = qd_all.shape[0]
    ids = np.full((nq, k), -1, dtype=np.int64)
    dists = np.full((nq, k), np.inf)
    n_cand = np.zeros(nq, dtype=np.int64)
    n_s1 = np.zeros(nq, dtype=np.int64)
    n_s2 = np.zeros(nq, dtype=np.int64)
    margin = np.full(nq, np.inf)
    for qi in range(nq):
        qd, qr = qd_all[qi], qr_all[qi]
        lists, g = probe(idx, qd, nprobe)
        gs = np.sort(g)
        mg = math.inf
        if nprobe < idx.nlist:
            mg = (gs[nprobe] - gs[nprobe - 1]) / max(gs[nprobe], 1e-30)
        two = refine and idx.bits > 1
        pos, lb, ub, sc, la, ua, sca = [], [], [], [], [], [], []
        for j in lists:
            e = estimate_list(idx, int(j), qd, float(g[j]), qr2_all[qi], sig_all[qi], eps0, m, qbits)
            sl = idx.list_slice(int(j))
            pos.append(np.arange(sl.start, sl.stop))
            lb.append(e["lb"]); ub.append(e["ub"]); sc.append(np.maximum(np.abs(e["dis"]), e["scale"]))
            if two:
                e1 = estimate_list(idx, int(j), qd, float(g[j]), qr2_all[qi], sig_all[qi], eps0, m,
                                   qbits, sign_plane=True)
                la.append(e1["lb"]); ua.append(e1["ub"])
                sca.append(np.maximum(np.abs(e1["dis"]), e1["scale"]))
        pos = np.concatenate(pos) if pos else np.zeros(0, dtype=np.int64)
        lb = np.concatenate(lb) if lb else np.zeros(0)
        ub = np.concatenate(ub) if ub else np.zeros(0)
        sc = np.concatenate(sc) if sc else np.zeros(0)
        n_cand[qi] = pos.size
        if two:                                             # 1 bit + refinement
            la, ua, sca = np.concatenate(la), np.concatenate(ua), np.concatenate(sca)
            tau_a1 = _kth(ua, k)
            s1a = la <= tau_a1
            tau_a = min(tau_a1, _kth(ub[s1a], k)) if s1a.any() else tau_a1
            s1 = s1a & (lb <= tau_a)                        # stage-1 survivors
        else:
            tau_a = _kth(ub, k)
            s1 = lb <= tau_a                                # stage-1 survivors
        # stage-2 quantities (Eq. 7) of every candidate, used on S1 only
        diso = idx.xnorm2[pos] + qp2_all[qi] - 2.0 * (idx.xd[pos] @ qd)
        lb2 = diso - m * sig_all[qi]
        ub2 = diso + m * sig_all[qi]
        sc2 = np.maximum(np.abs(diso), idx.xnorm2[pos] + qp2_all[qi])
        if mode == MODE_MRQ_PLUS and s1.any():
            kth_ub2 = _kth(ub2[s1], k)
            tau_b = min(tau_a, kth_ub2)
            s2 = s1 & (lb2 <= tau_b)
        else:
            kth_ub2, tau_b = math.inf, math.inf
            s2 = s1
        n_s1[qi] = int(s1.sum())
        p2 = pos[s2]
        n_s2[qi] = p2.size
        ex_all = (np.sum((idx.xd[pos] - qd) ** 2, axis=1)
                  + np.sum((idx.xr[pos] - qr) ** 2, axis=1))
        if p2.size:
            ex = ex_all[s2]
            oid = idx.ids[p2]
            o = np.lexsort((oid, ex))
            kk = min(k, p2.size)
            ids[qi, :kk] = oid[o[:kk]]
            dists[qi, :kk] = ex[o[:kk]]
            srt = ex[o]
            if srt.size > 1:
                lim = min(k + 1, srt.size)
                gaps = np.diff(srt[:lim]) / np.maximum(srt[1:lim], 1e-30)
                mg = min(mg, float(np.min(gaps)))
            dk = srt[kk - 1] if p2.size >= k else math.inf
        else:
            dk = math.inf
        in_ans = np.isin(idx.ids[pos], ids[qi, :min(k, p2.size)])
        near = in_ans | (ex_all <= dk * (1 + 1e-6))
        rel1 = near | ((mode == MODE_MRQ_PLUS) & (ub2 <= kth_ub2 * (1 + 1e-6)))
        if two:
            # the sign-plane level: its test of an answer-relevant candidate, and the
            # candidates whose upper bounds set tau_A' or tau_A
            rel1a = rel1 | (ua <= tau_a1 * (1 + 1e-6)) | (ub <= tau_a * (1 + 1e-6))
            if pos.size and math.isfinite(tau_a1) and rel1a.any():
                mg = min(mg, _decision_margin(la, ua, sca, tau_a1, k, rel1a))
            rel1 = rel1 & s1a
            if rel1.any() and math.isfinite(tau_a):
                mg = min(mg, _decision_margin(lb[s1a], ub[s1a], sc[s1a], tau_a, k, rel1[s1a]))
        elif pos.size and math.isfinite(tau_a) and rel1.any():
            mg = min(mg, _decision_margin(lb, ub, sc, tau_a, k, rel1))
        rel2 = near & s1
        if mode == MODE_MRQ_PLUS and math.isfinite(tau_b) and rel2.any():
            mg = min(mg, _decision_margin(lb2[s1], ub2[s1], sc2[s1], tau_b, k, rel2[s1]))
        margin[qi] = mg
    return SearchResult(ids, dists, n_cand, n_s1, n_s2, margin)


def sq8_train(xd):
    """MR-SQ (Appendix A.2, Exp-5): 8-bit scalar quantization of the projected lead
    coordinates (the stored x_d' rows) instead of RaBitQ codes.

    Reading (the paper only names "8-bit SQ"): per dimension a uniform grid of 256 levels
    from the column's minimum to its maximum over the base, delta = (hi - lo) / 255;
    code c = floor((x - lo) / delta + 1/2) clamped to [0, 255], reconstruction
    x_hat = lo + c * delta.  A constant column (delta = 0) gets code 0.  The grid and
    the code decision are taken in float32 (the GPU kernel's precision).
    Returns lo (float32 [d]), delta (float32 [d]), codes (uint8 [n x d]).
    """
    X = np.asarray(xd, dtype=np.float32)
    lo = X.min(axis=0)
    hi = X.max(axis=0)
    delta = ((hi - lo) / np.float32(255)).astype(np.float32)
    safe = np.where(delta > 0, delta, np.float32(1))
    t = ((X - lo) / safe).astype(np.float32)
    c = np.floor(t + np.float32(0.5))
    c = np.where(delta > 0, np.clip(c, 0, 255), 0).astype(np.uint8)
    return lo, delta, c


def sq8_estimate(idx: OracleIndex, sq, qd, qr2, pos=None):
    """MR-SQ estimate (Exp-5) of the rows ``pos`` (all rows when None) for one projected
    query: dis'' = |q_d' - x_hat|^2 + |x_r|^2 + |q_r|^2 with x_hat the SQ8
    reconstruction; the residual inner product is dropped, as in Eq. 4."""
    lo, delta, codes = sq
    sel = slice(None) if pos is None else pos
    xhat = lo.astype(np.float64) + codes[sel].astype(np.float64) * delta.astype(np.float64)
    xr = idx.xr[sel]
    return np.sum((qd - xhat) ** 2, axis=1) + np.sum(xr * xr, axis=1) + qr2


def _search_rerank(idx: OracleIndex, Q, k: int, nprobe: int, rerank: int,
                   estimate) -> SearchResult:
    """The fixed-rerank-range search of Exp-5 (MR-SQ, MR-PQ): after the projection and
    probe of Algorithm 2, the `rerank` probed candidates with the smallest estimate
    ``estimate(qd, qr2, pos)`` (ties by id) get their exact distance, and the answer is
    the k smallest exact distances (ties by id).  n_s1 = n_s2 = the number reranked.
    ``margin``: the probe boundary, how far each answer-relevant candidate (exact
    distance within the k-th) sits from the rerank cut in the estimate, and
    consecutive answer distances around rank k."""
    qd_all, qr_all, qr2_all, _, _ = project_queries(idx, Q)
    nq = qd_all.shape[0]
    ids = np.full((nq, k), -1, dtype=np.int64)
    dists = np.full((nq, k), np.inf)
    n_cand = np.zeros(nq, dtype=np.int64)
    n_rr = np.zeros(nq, dtype=np.int64)
    margin = np.full(nq, np.inf)
    for qi in range(nq):
        qd, qr = qd_all[qi], qr_all[qi]
        lists, g = probe(idx, qd, nprobe)
        gs = np.sort(g)
        mg = math.inf
        if nprobe < idx.nlist:
            mg = (gs[nprobe] - gs[nprobe - 1]) / max(gs[nprobe], 1e-30)
        pos = (np.concatenate([np.arange(idx.list_offsets[j], idx.list_offsets[j + 1])
                               for j in lists]) if len(lists) else np.zeros(0, dtype=np.int64))
        n_cand[qi] = pos.size
        if pos.size == 0:
            margin[qi] = mg
            continue
        est = estimate(qd, qr2_all[qi], pos)
        order = np.lexsort((idx.ids[pos], est))
        R = min(rerank, pos.size)
        sel = order[:R]
        n_rr[qi] = R
        ex_all = (np.sum((idx.xd[pos] - qd) ** 2, axis=1)
                  + np.sum((idx.xr[pos] - qr) ** 2, axis=1))
        ex = ex_all[sel]
        oid = idx.ids[pos[sel]]
        o = np.lexsort((oid, ex))
        kk = min(k, R)
        ids[qi, :kk] = oid[o[:kk]]
        dists[qi, :kk] = ex[o[:kk]]
        srt = ex[o]
        if srt.size > 1:
            lim = min(k + 1, srt.size)
            gaps = np.diff(srt[:lim]) / np.maximum(srt[1:lim], 1e-30)
            mg = min(mg, float(np.min(gaps)))
        if R < pos.size:
            dk = srt[kk - 1]
            rel = ex_all <= dk * (1 + 1e-6)           # could be in the answer
            inside = np.zeros(pos.size, dtype=bool)
            inside[sel] = True
            t_in, t_out = est[order[R - 1]], est[order[R]]
            for i in np.nonzero(rel)[0]:
                if inside[i]:
                    mg = min(mg, (t_out - est[i]) / max(t_out, 1e-30))
                else:
                    mg = min(mg, (est[i] - t_in) / max(est[i], 1e-30))
        margin[qi] = mg
    return SearchResult(ids, dists, n_cand, n_rr, n_rr.copy(), margin)




def search_mrsq8(idx: OracleIndex, Q, k: int, nprobe: int, rerank: int = 500,
                 sq=None) -> SearchResult:
    """MR-SQ search (Exp-5): SQ8 estimates over the probed lists, then a fixed rerank
    range instead of an error bound (``_search_rerank``), with
      dis'' = |q_d' - x_hat|^2 + |x_r|^2 + |q_r|^2   (the residual inner product
              -2<x_r, q_r> is dropped, as Eq. 4 drops it).
    """
    sq = sq if sq is not None else sq8_train(idx.xd)
    return _search_rerank(idx, Q, k, nprobe, rerank,
                          lambda qd, qr2, pos: sq8_estimate(idx, sq, qd, qr2, pos))


def opq_train(X, M: int, K: int, init_idx, opq_iters: int = 4, km_iters: int = 6):
    """MR-PQ (Appendix A.2, Exp-5): optimized product quantization of the projected lead
    coordinates (rows of X, n x d).

    Reading (the paper names OPQ only): the non-parametric OPQ of Ge et al. (2013) --
    alternate, ``opq_iters`` times, (a) Lloyd k-means (``km_iters`` rounds, warm
    started) of each of the M subspaces of d/M consecutive coordinates of X R into K
    centroids, and (b) the orthogonal R minimising |X R - Y|_F for the decoded Y, which
    is U V^T for the SVD X^T Y = U S V^T (orthogonal Procrustes); then a final k-means
    round set and the codes.  R starts at the identity; the initial centroids of every
    subspace are the rows ``init_idx`` (K of them).
    Returns R (d x d), codebooks (M x K x d/M), codes (uint8 n x M).
    """
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if d % M or K > n or K > 256:
        raise ValueError("invalid PQ shape")
    ds = d // M
    R = np.eye(d)
    Xr = X @ R
    C = np.stack([Xr[np.asarray(init_idx), m * ds:(m + 1) * ds] for m in range(M)])
    codes = np.zeros((n, M), dtype=np.int64)
    for _ in range(opq_iters):
        Xr = X @ R
        for m in range(M):
            C[m], codes[:, m] = kmeans(Xr[:, m * ds:(m + 1) * ds], C[m], km_iters)
        Y = pq_decode(C, codes)
        U, _, Vt = np.linalg.svd(X.T @ Y)
        R = U @ Vt
    Xr = X @ R
    for m in range(M):
        C[m], codes[:, m] = kmeans(Xr[:, m * ds:(m + 1) * ds], C[m], km_iters)
    return R, C, codes.astype(np.uint8)


def pq_decode(C, codes):
    """Concatenated centroids of the codes (n x d, in the rotated frame X R)."""
    return np.concatenate([C[m][codes[:, m]] for m in range(C.shape[0])], axis=1)


def pq_estimate(idx: OracleIndex, pq, qd, qr2, pos=None):
    """MR-PQ estimate (asymmetric distance computation): with q' = q_d' R and the
    lookup table T[m][j] = |q'_m - C[m][j]|^2 of each subspace m,
    dis'' = sum_m T[m][code_m] + |x_r|^2 + |q_r|^2 (the residual cross term dropped)."""
    R, C, codes = pq
    sel = slice(None) if pos is None else pos
    M, K, ds = C.shape
    qp = np.asarray(qd, dtype=np.float64) @ R
    T = np.stack([np.sum((qp[m * ds:(m + 1) * ds][None, :] - C[m]) ** 2, axis=1)
                  for m in range(M)])                       # M x K
    cs = codes[sel].astype(np.int64)
    lead = np.sum(T[np.arange(M)[None, :], cs], axis=1)
    xr = idx.xr[sel]
    return lead + np.sum(xr * xr, axis=1) + qr2


def search_mrpq(idx: OracleIndex, Q, k: int, nprobe: int, pq, rerank: int = 500) -> SearchResult:
    """MR-PQ search (Exp-5): OPQ estimates (``pq`` from ``opq_train`` on idx.xd) over the
    probed lists and the fixed rerank range of ``_search_rerank``."""
    return _search_rerank(idx, Q, k, nprobe, rerank,
                          lambda qd, qr2, pos: pq_estimate(idx, pq, qd, qr2, pos))


def search_literal(idx: OracleIndex, Q, k: int, nprobe: int, *, eps0: float = 1.9,
                   m: float = 4.0, mode: int = MODE_MRQ_PLUS, qbits: int = 0) -> SearchResult:
    """Algorithm 2 exactly as printed: probed lists in ascending centroid distance,
    members in stored order, tau = the k-th exact distance held in the result
    queue (+inf until it holds k); a candidate reaches the exact distance only if
    dis' - eps_b - eps_r < tau and (MRQ+) dis_o' - eps_r < tau (Eq. 7)."""
    qd_all, qr_all, qr2_all, sig_all, qp2_all = project_queries(idx, Q)
    nq = qd_all.shape[0]
    ids = np.full((nq, k), -1, dtype=np.int64)
    dists = np.full((nq, k), np.inf)
    n_cand = np.zeros(nq, dtype=np.int64)
    n_s1 = np.zeros(nq, dtype=np.int64)
    n_s2 = np.zeros(nq, dtype=np.int64)
    for qi in range(nq):
        qd, qr = qd_all[qi], qr_all[qi]
        lists, g = probe(idx, qd, nprobe)
        heap_d: list[float] = []
        heap_i: list[int] = []
        for j in lists:
            e = estimate_list(idx, int(j), qd, float(g[j]), qr2_all[qi], sig_all[qi], eps0, m, qbits)
            sl = idx.list_slice(int(j))
            for t, p in enumerate(range(sl.start, sl.stop)):
                n_cand[qi] += 1
                tau = heap_d[k - 1] if len(heap_d) >= k else math.inf
                if not e["lb"][t] < tau:
                    continue
                n_s1[qi] += 1
                if mode == MODE_MRQ_PLUS:
                    diso = idx.xnorm2[p] + qp2_all[qi] - 2.0 * float(idx.xd[p] @ qd)
                    if not diso - m * sig_all[qi] < tau:
                        continue
                n_s2[qi] += 1
                ex = float(np.sum((idx.xd[p] - qd) ** 2) + np.sum((idx.xr[p] - qr) ** 2))
                oid = int(idx.ids[p])
                at = 0
                while at < len(heap_d) and (heap_d[at], heap_i[at]) < (ex, oid):
                    at += 1
                heap_d.insert(at, ex)
                heap_i.insert(at, oid)
                del heap_d[k:], heap_i[k:]
        ids[qi, :len(heap_i)] = heap_i
        dists[qi, :len(heap_d)] = heap_d
    return SearchResult(ids, dists, n_cand, n_s1, n_s2, np.full(nq, np.inf))


def exact_knn(S, Q, k: int, block: int = 4096):
    """Brute-force exact k-NN under squared Euclidean distance (Section 2.1), FP64,
    ties by id.  Returns (ids, dists)."""
    S = np.asarray(S, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    s2 = np.sum(S * S, axis=1)
    ids = np.empty((Q.shape[0], k), dtype=np.int64)
    dists = np.empty((Q.shape[0], k))
    for a in range(0, Q.shape[0], block):
        q = Q[a:a + block]
        dd = s2[None, :] + np.sum(q * q, axis=1)[:, None] - 2.0 * (q @ S.T)
        kk = min(S.shape[0], k + 64)
        cand = np.argpartition(dd, kk - 1, axis=1)[:, :kk]
        for r in range(q.shape[0]):
            c = cand[r]
            ex = np.sum((S[c] - q[r]) ** 2, axis=1)      # direct recheck of the candidates
            o = np.lexsort((c, ex))[:k]
            ids[a + r] = c[o]
            dists[a + r] = ex[o]
    return ids, dists


def recall_at_k(found: np.ndarray, truth: np.ndarray) -> float:
    """Recall@k = |T intersect G| / |G| averaged over queries (Section 2.1)."""
    k = truth.shape[1]
    hit = 0
    for f, t in zip(found, truth):
        hit += len(set(f[:k].tolist()) & set(t.tolist()))
    return hit / truth.size
