"""Seeded synthetic inputs shaped like matrix-factorisation embeddings.

This module only draws random numbers. It holds none of the reverse k-MIPS
arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path can be fed
from it without sharing any of the method's code.

Recipe (stands in for the MovieLens / Netflix / Amazon / Yahoo! MF vectors of
the paper's Section 5.1, which are not available here):

* every vector is ``x = s * g / ||g||`` with ``g ~ N(0, I_d / d)`` and a
  per-vector norm ``s ~ LogNormal(0, 0.5)``, so ``||x||`` is lognormal;
* Q (users) and P (items) are drawn independently from one PCG64 stream,
  Q first, then P;
* queries "from P" are bit copies of P rows chosen without replacement with
  the stream seeded ``seed + 1000`` (Section 5.1 draws its 1,000 queries from
  P);
* "random" queries are plain ``N(0, I_d / d)`` vectors (seed ``seed + 2000``).

All arrays are C-contiguous little-endian float32 ``[rows][d]``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["mf_like", "make_problem", "queries_from_items", "random_queries",
           "integer_problem", "CONFIGS"]


def mf_like(rng: np.random.Generator, rows: int, d: int, sigma: float = 0.5) -> np.ndarray:
    """``rows`` vectors ``s * g/||g||`` with lognormal norms ``s``."""
    out = np.empty((rows, d), dtype=np.float32)
    step = 1 << 18
    for r0 in range(0, rows, step):
        r1 = min(rows, r0 + step)
        g = rng.standard_normal((r1 - r0, d)) / np.sqrt(d)
        s = rng.lognormal(0.0, sigma, size=r1 - r0)
        gn = np.sqrt(np.einsum("ij,ij->i", g, g))
        gn[gn == 0.0] = 1.0
        out[r0:r1] = (g * (s / gn)[:, None]).astype(np.float32)
    return out


def make_problem(n: int, m: int, d: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """User matrix Q [n, d] and item matrix P [m, d] (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = mf_like(rng, n, d)
    P = mf_like(rng, m, d)
    return Q, P


def queries_from_items(P: np.ndarray, nq: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """``nq`` distinct rows of P (bit copies) and their row indices."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    idx = rng.choice(P.shape[0], size=min(nq, P.shape[0]), replace=False)
    if nq > P.shape[0]:
        idx = np.concatenate([idx, rng.integers(0, P.shape[0], nq - P.shape[0])])
    return np.ascontiguousarray(P[idx]), idx.astype(np.int64)


def random_queries(nq: int, d: int, seed: int) -> np.ndarray:
    """``nq`` query vectors drawn from ``N(0, I_d / d)``."""
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    return (rng.standard_normal((nq, d)) / np.sqrt(d)).astype(np.float32)


def random_ks(nq: int, k_lo: int, k_hi: int, seed: int) -> np.ndarray:
    """Per-query k drawn uniformly from ``[k_lo, k_hi]`` (int32)."""
    rng = np.random.Generator(np.random.PCG64(seed + 3000))
    return rng.integers(k_lo, k_hi + 1, size=nq).astype(np.int32)


def integer_problem(n: int, m: int, d: int, seed: int, lim: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """Small-integer vectors (components in ``[-lim, lim]``).

    Every inner product of such vectors is an exact small integer in float32,
    so ties between items are frequent and exact on every precision path.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = rng.integers(-lim, lim + 1, size=(n, d)).astype(np.float32)
    P = rng.integers(-lim, lim + 1, size=(m, d)).astype(np.float32)
    return Q, P


# Workload shapes of the five configurations (users n, items m, dimension d).
CONFIGS = {
    "tiny": dict(n=2_000, m=1_000, d=50, k_max=25, k=10, nq=100, seed=0),
    "plain": dict(n=100_000, m=50_000, d=50, k_max=25, ks=(1, 5, 10, 15, 20, 25), nq=1_000, seed=1),
    "precision": dict(n=500_000, m=100_000, d=64, k_max=25, k=10, nq=2_000, seed=2),
    "batching": dict(n=1_000_000, m=500_000, d=50, k_max=25, k_range=(1, 25), nq=10_000, seed=3),
    "serving": dict(n=1_000_000, m=500_000, d=50, k_max=25, k_range=(1, 25), seed=4),
}
