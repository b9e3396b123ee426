"""Seeded synthetic workloads for MRQ (approximate k-NN with PCA projection plus quantization).

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the method itself (no PCA, no clustering, no quantization, no
distance estimate): only random draws and the data recipe.

Recipe (a stand-in for the paper's datasets, Table 1; the paper's own data is
not available here).  The paper observes that after PCA the per-dimension
variance of real embeddings is long-tailed (Section 3.2, Fig. 2); the recipe
reproduces that spectrum explicitly:

* ``U`` is a Haar-random D x D orthogonal matrix (QR of a Gaussian matrix with
  the signs of diag(R) made positive).
* ``lam[i] = (i+1) ** -alpha`` for i = 0..D-1.
* Mixture centres ``m_j = U diag(sqrt(lam)) z_j`` with ``z_j ~ N(0, I)``.
* A point of component j is ``m_j + spread * U diag(sqrt(lam * f_j)) g`` with
  ``g ~ N(0, I)``; ``f_j`` is 1 (isotropic components) or a per-axis
  log-normal(0, 0.5) factor (anisotropic, embedding-like workload).
* Components are drawn uniformly; queries are fresh draws from the same
  mixture (never base points).
* Optionally every vector is scaled to unit norm (embedding-like workload).

Seeds: ``1000 * workload_id + {0: basis, 1: base, 2: queries, 3: mixture,
4: method draws}``; numpy's PCG64 is platform-independent, so the same seed
gives the same draws on x86_64 and aarch64 (BLAS rounding may differ in the
last bit between machines; nothing here depends on that).

Random numbers the method itself draws (the Gaussian matrix behind the random
rotation P_r of Algorithm 1, the seeded permutation that picks the initial IVF
centroids) are produced here too, so that the oracle and the GPU library can be
fed identical draws.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "workload",
    "spectrum",
    "haar_orthogonal",
    "make_mixture",
    "sample",
    "base_and_queries",
    "rotation_gaussian",
    "kmeans_init_indices",
    "zipf_list_sizes",
    "zipf_clustered",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic workload (sizes and the spectrum exponent)."""

    wid: int
    name: str
    n: int
    D: int
    n_comp: int
    alpha: float
    n_query: int
    d: int
    bits: int
    nlist: int
    nprobe: int
    k: int
    spread: float = 0.5
    anisotropic: bool = False
    unit_norm: bool = False

    def seed(self, what: str) -> int:
        off = {"basis": 0, "base": 1, "queries": 2, "mixture": 3, "method": 4}[what]
        return 1000 * self.wid + off

    def scaled(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# The five workload shapes the hot path is exercised on.
WORKLOADS = {
    # small plain case: the oracle finishes it in seconds
    "small": Workload(1, "small-20k-d128", n=20_000, D=128, n_comp=64, alpha=1.2,
                      n_query=200, d=32, bits=1, nlist=64, nprobe=8, k=10),
    # GIST-like shape (D=960, 1M, 4096 lists)
    "gist": Workload(2, "gist-like-1M-d960", n=1_000_000, D=960, n_comp=1024, alpha=1.0,
                     n_query=10_000, d=128, bits=1, nlist=4096, nprobe=64, k=10),
    # embedding-like, anisotropic, unit-normalised
    "embed": Workload(3, "embedding-like-1M-d768", n=1_000_000, D=768, n_comp=2048,
                      alpha=0.8, n_query=10_000, d=128, bits=1, nlist=4096, nprobe=64,
                      k=10, anisotropic=True, unit_norm=True),
    # DEEP-like with Zipf list sizes
    "deep": Workload(4, "deep-like-10M-d96-zipf", n=10_000_000, D=96, n_comp=4096,
                     alpha=1.5, n_query=100_000, d=32, bits=4, nlist=16_384, nprobe=64,
                     k=10),
    # MSMARCO-like shape, serving
    "serve": Workload(5, "msmarco-like-5M-d1024", n=5_000_000, D=1024, n_comp=4096,
                      alpha=1.0, n_query=10_000, d=256, bits=2, nlist=4096, nprobe=64,
                      k=10),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return w.scaled(**overrides) if overrides else w


def spectrum(D: int, alpha: float) -> np.ndarray:
    """Power-law variance profile lam[i] = (i+1)^-alpha (float64)."""
    return np.arange(1, D + 1, dtype=np.float64) ** (-alpha)


def haar_orthogonal(D: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random orthogonal matrix (float64): QR of a Gaussian, sign-fixed."""
    g = rng.standard_normal((D, D))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


@dataclasses.dataclass
class Mixture:
    U: np.ndarray          # D x D float64
    lam: np.ndarray        # D float64
    centres: np.ndarray    # n_comp x D float64
    axis_scale: np.ndarray  # n_comp x D float64 (per-axis std multipliers in the U frame)
    spread: float
    unit_norm: bool


def make_mixture(w: Workload) -> Mixture:
    """Mixture parameters of a workload (deterministic in its seeds)."""
    U = haar_orthogonal(w.D, np.random.default_rng(w.seed("basis")))
    lam = spectrum(w.D, w.alpha)
    rng = np.random.default_rng(w.seed("mixture"))
    z = rng.standard_normal((w.n_comp, w.D))
    centres = (z * np.sqrt(lam)[None, :]) @ U.T
    if w.anisotropic:
        f = np.exp(rng.normal(0.0, 0.5, size=(w.n_comp, w.D)))
    else:
        f = np.ones((w.n_comp, w.D))
    axis_scale = np.sqrt(lam[None, :] * f)
    return Mixture(U=U, lam=lam, centres=centres, axis_scale=axis_scale,
                   spread=w.spread, unit_norm=w.unit_norm)


def sample(mix: Mixture, n: int, seed: int, chunk: int = 65536,
           comp: np.ndarray | None = None) -> np.ndarray:
    """Draw n float32 points from the mixture (chunked to bound host memory)."""
    rng = np.random.default_rng(seed)
    D = mix.U.shape[0]
    if comp is None:
        comp = rng.integers(0, mix.centres.shape[0], size=n)
    out = np.empty((n, D), dtype=np.float32)
    Ut = mix.U.T.astype(np.float32)
    centres32 = mix.centres.astype(np.float32)
    scale32 = mix.axis_scale.astype(np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        c = comp[s:e]
        g = rng.standard_normal((e - s, D), dtype=np.float32)
        g *= scale32[c] * np.float32(mix.spread)
        x = g @ Ut
        x += centres32[c]
        if mix.unit_norm:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = x
    return out


def base_and_queries(w: Workload, n: int | None = None, n_query: int | None = None):
    """(base, queries) float32 arrays of a workload; n / n_query override sizes."""
    mix = make_mixture(w)
    base = sample(mix, w.n if n is None else n, w.seed("base"))
    queries = sample(mix, w.n_query if n_query is None else n_query, w.seed("queries"))
    return base, queries


def rotation_gaussian(d: int, seed: int) -> np.ndarray:
    """d x d standard-normal float64 draw behind the random rotation P_r (Alg. 1)."""
    return np.random.default_rng(seed).standard_normal((d, d))


def kmeans_init_indices(n: int, nlist: int, seed: int) -> np.ndarray:
    """First nlist entries of a seeded permutation of the base (IVF initialisation)."""
    return np.random.default_rng(seed).permutation(n)[:nlist].astype(np.int64)


def zipf_list_sizes(n: int, nlist: int, s: float, seed: int) -> np.ndarray:
    """Rank-size Zipf list sizes size_l ~ l^-s (shuffled), each >= 1, summing to n."""
    rng = np.random.default_rng(seed)
    w = np.arange(1, nlist + 1, dtype=np.float64) ** (-s)
    sizes = np.maximum(1, np.floor(w / w.sum() * n)).astype(np.int64)
    short = n - int(sizes.sum())
    if short > 0:
        sizes[:short % nlist] += 1
        sizes += short // nlist
    elif short < 0:
        i = 0
        while short < 0:
            take = min(-short, int(sizes[i]) - 1)
            sizes[i] -= take
            short += take
            i += 1
    rng.shuffle(sizes)
    return sizes


def zipf_clustered(w: Workload, n: int, nlist: int, s: float = 1.1, spread: float = 0.25):
    """Base whose IVF lists have Zipf(s) sizes: every list is generated around its own
    centre (a draw from the mixture).  Returns (base float32, centres float32 nlist x D,
    sizes int64)."""
    mix = make_mixture(w)
    centres = sample(mix, nlist, w.seed("method") + 17)
    sizes = zipf_list_sizes(n, nlist, s, w.seed("method") + 18)
    rng = np.random.default_rng(w.seed("base"))
    D = w.D
    base = np.empty((n, D), dtype=np.float32)
    Ut = mix.U.T.astype(np.float32)
    sc = (np.sqrt(mix.lam) * spread).astype(np.float32)
    pos = 0
    order = rng.permutation(n)
    owner = np.repeat(np.arange(nlist), sizes)
    chunk = 65536
    for s0 in range(0, n, chunk):
        e = min(n, s0 + chunk)
        idx = order[s0:e]
        g = rng.standard_normal((e - s0, D), dtype=np.float32) * sc[None, :]
        base[idx] = g @ Ut + centres[owner[s0:e]]
        pos = e
    return base, centres, sizes
