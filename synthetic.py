"""Seeded synthetic workloads for range-filtered k-NN search.

This module only draws random inputs: base vectors, their numeric attributes,
query vectors, query rank ranges and per-query k. It holds none of the search
method's arithmetic, so both the CPU oracle (``oracle/``) and the GPU library
(``paper_2504_04018_gb300``) can consume the same inputs without sharing code.

Every generator is deterministic in its seed (NumPy ``PCG64``). Vectors are
drawn in float64 and stored as float32; consumers that work in float64 promote
the stored float32 values.

Workload shapes stand in for the datasets of the paper's experiments (SIFT
d=128, DEEP d=96, 1M points; Table 3) and for its query-range families: random
"mix" ranges and fixed fractions 2^-j of N (Section 5.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def mixture_centers(n_comp: int, d: int, seed: int) -> np.ndarray:
    """Component centers drawn uniformly from [-1, 1]^d (float64)."""
    return _rng(seed).uniform(-1.0, 1.0, size=(n_comp, d))


def mixture_points(centers: np.ndarray, n: int, sigma: float, seed: int,
                   normalise: bool = False) -> np.ndarray:
    """n points of an isotropic Gaussian mixture with the given centers.

    A point is ``centers[c] + sigma * z`` with ``c`` uniform over the
    components and ``z ~ N(0, I_d)``; optionally L2-normalised. Returned as
    float32 (drawn in float64).
    """
    rng = _rng(seed)
    comp = rng.integers(0, centers.shape[0], size=n)
    out = np.empty((n, centers.shape[1]), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        x = centers[comp[s:e]] + sigma * rng.standard_normal((e - s, centers.shape[1]))
        if normalise:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = x
    return out


def anisotropic_points(n: int, d: int, exponent: float, seed: int,
                       basis_seed: int) -> np.ndarray:
    """Gaussian with a power-law spectrum, L2-normalised (float32).

    ``x = U diag(i^(-exponent/2)) z`` with ``z ~ N(0, I)`` and ``U`` a random
    orthogonal matrix (QR of a Gaussian matrix drawn from ``basis_seed``), so
    the covariance eigenvalues decay as ``i^-exponent``.
    """
    g = _rng(basis_seed).standard_normal((d, d))
    u, rr = np.linalg.qr(g)
    u = u * np.sign(np.diag(rr))[None, :]
    scale = np.arange(1, d + 1, dtype=np.float64) ** (-exponent / 2.0)
    rng = _rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 15
    for s in range(0, n, step):
        e = min(n, s + step)
        z = rng.standard_normal((e - s, d)) * scale[None, :]
        x = z @ u.T
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = x
    return out


def permutation_attributes(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1, as float64 attribute values."""
    return _rng(seed).permutation(n).astype(np.float64)


def ranges_from_fractions(n: int, fracs: np.ndarray, seed: int):
    """Inclusive 0-based rank ranges [l, r] of width max(1, round(frac * n)).

    The left end is uniform over the positions where the range fits.
    Returns int64 arrays (l, r).
    """
    rng = _rng(seed)
    w = np.maximum(1, np.rint(np.asarray(fracs, dtype=np.float64) * n)).astype(np.int64)
    w = np.minimum(w, n)
    l = rng.integers(0, n - w + 1).astype(np.int64)
    return l, l + w - 1


def log_uniform_fractions(nq: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """nq fractions with log-uniform distribution on [lo, hi]."""
    rng = _rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=nq))


@dataclasses.dataclass
class Workload:
    """One seeded workload: base set, attributes, queries, ranges and k."""
    name: str
    base: np.ndarray          # float32 [N, d], original order
    attr: np.ndarray          # float64 [N]
    queries: np.ndarray       # float32 [nq, d]
    l: np.ndarray             # int64 [nq], inclusive rank range (after re-ranking)
    r: np.ndarray             # int64 [nq]
    k: np.ndarray             # int32 [nq]
    metric: str               # "l2" (squared Euclidean) or "ip" (negative inner product)
    M: int                    # graph degree parameter (cap on out-degree is 2*M)
    ef: int                   # default beam width
    leaf_size: int = 256

    @property
    def n(self) -> int:
        return self.base.shape[0]

    @property
    def d(self) -> int:
        return self.base.shape[1]


def _mixture_workload(name, n, d, n_comp, nq, fracs_fn, cfg, metric, M, ef,
                      normalise=False, k_fn=None, sigma=0.1):
    centers = mixture_centers(n_comp, d, 1000 + cfg)
    base = mixture_points(centers, n, sigma, 1000 + cfg + 100, normalise)
    queries = mixture_points(centers, nq, sigma, 2000 + cfg, normalise)
    attr = permutation_attributes(n, 3000 + cfg)
    fracs = fracs_fn(nq)
    l, r = ranges_from_fractions(n, fracs, 2000 + cfg + 500)
    k = k_fn(nq) if k_fn is not None else np.full(nq, 10, dtype=np.int32)
    return Workload(name, base, attr, queries, l, r, k.astype(np.int32), metric, M, ef)


def tiny(n: int = 10_000, nq: int = 200, d: int = 128) -> Workload:
    """N=10^4, d=128 L2, 64-component mixture; widths uniform over
    {1, 5, 10, 25, 50, 100}% of N; k=10, ef=64, M=16."""
    choices = np.array([0.01, 0.05, 0.10, 0.25, 0.50, 1.0])
    fr = lambda q: choices[_rng(2001 + 600).integers(0, len(choices), size=q)]
    return _mixture_workload("tiny", n, d, 64, nq, fr, 1, "l2", 16, 64)


def scale(n: int = 1_000_000, nq: int = 10_000, d: int = 128, n_comp: int = 1024) -> Workload:
    """N=10^6, d=128 L2, 1,024-component mixture; widths 2^-j N for j=0..10
    (equal share per j); k=10; M=32."""
    def fr(q):
        j = np.arange(q) % 11
        return 2.0 ** (-j.astype(np.float64))
    return _mixture_workload("scale", n, d, n_comp, nq, fr, 2, "l2", 32, 64)


def training_queries(wl: Workload, nq: int, n_comp: int, seed: int, sigma: float = 0.1):
    """Extra queries from the same mixture as `wl` (its centers are redrawn
    from the workload's seed) with range widths drawn like wl's (resampled
    from its width distribution), for training a search-budget predictor.
    Returns (queries float32 [nq, d], l, r int64 [nq])."""
    cfg = {"tiny": 1, "scale": 2, "precision": 3, "batching": 4}[wl.name]
    centers = mixture_centers(n_comp, wl.d, 1000 + cfg)
    q = mixture_points(centers, nq, sigma, seed, normalise=(wl.metric == "ip"))
    widths = (wl.r - wl.l + 1).astype(np.float64) / wl.n
    fr = _rng(seed + 1).choice(widths, size=nq)
    l, r = ranges_from_fractions(wl.n, fr, seed + 2)
    return q, l, r


def precision(n: int = 1_000_000, nq: int = 10_000, d: int = 96, n_comp: int = 1024) -> Workload:
    """N=10^6, d=96 unit-normalised mixture, inner product; log-uniform
    widths 0.1%-100%; k=10; M=32."""
    fr = lambda q: log_uniform_fractions(q, 1e-3, 1.0, 2003 + 600)
    return _mixture_workload("precision", n, d, n_comp, nq, fr, 3, "ip", 32, 64, normalise=True)


def batching(n: int = 10_000_000, nq: int = 100_000, d: int = 96, n_comp: int = 1024) -> Workload:
    """N=10^7, d=96 unit-normalised mixture, inner product; log-uniform
    widths 0.01%-100%; k uniform over {1, 10, 100}; M=32."""
    fr = lambda q: log_uniform_fractions(q, 1e-4, 1.0, 2004 + 600)
    kf = lambda q: np.array([1, 10, 100], dtype=np.int32)[_rng(2004 + 700).integers(0, 3, size=q)]
    return _mixture_workload("batching", n, d, n_comp, nq, fr, 4, "ip", 32, 64,
                             normalise=True, k_fn=kf)


def learned(n: int = 1_000_000, nq: int = 10_000, d: int = 768, n_train: int = 50_000) -> Workload:
    """N=10^6, d=768 anisotropic (power-law spectrum, exponent 1), L2-normalised,
    inner product; log-uniform widths 0.1%-100%; k=10; M=32. The first
    ``n_train`` queries are the training split, the rest held out."""
    base = anisotropic_points(n, d, 1.0, 1005, 1005 + 50)
    queries = anisotropic_points(n_train + nq, d, 1.0, 2005, 1005 + 50)
    attr = permutation_attributes(n, 3005)
    fr = log_uniform_fractions(n_train + nq, 1e-3, 1.0, 2005 + 600)
    l, r = ranges_from_fractions(n, fr, 2005 + 500)
    k = np.full(n_train + nq, 10, dtype=np.int32)
    return Workload("learned", base, attr, queries, l, r, k, "ip", 32, 64)


def small_mixture(n: int, d: int, nq: int, n_comp: int = 16, seed: int = 7,
                  metric: str = "l2", normalise: bool = False,
                  fracs: Optional[np.ndarray] = None, k: int = 10, M: int = 8,
                  ef: int = 32, leaf_size: int = 16) -> Workload:
    """A small mixture workload for unit tests (arbitrary seed and sizes)."""
    centers = mixture_centers(n_comp, d, seed)
    base = mixture_points(centers, n, 0.1, seed + 1, normalise)
    queries = mixture_points(centers, nq, 0.1, seed + 2, normalise)
    attr = permutation_attributes(n, seed + 3)
    if fracs is None:
        fracs = log_uniform_fractions(nq, max(1.0 / n, 1e-3), 1.0, seed + 4)
    l, r = ranges_from_fractions(n, fracs, seed + 5)
    wl = Workload("small", base, attr, queries, l, r, np.full(nq, k, dtype=np.int32),
                  metric, M, ef, leaf_size)
    return wl
