"""Graph generators: Chung-Lu power-law and R-MAT, finished into streams."""
from __future__ import annotations

import numpy as np

M32 = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def pack(u, v) -> np.ndarray:
    """Packed keys (min << 32) | max from two id arrays."""
    u = np.asarray(u, dtype=np.uint64)
    v = np.asarray(v, dtype=np.uint64)
    return (np.minimum(u, v) << S32) | np.maximum(u, v)


def unpack(keys: np.ndarray):
    keys = np.asarray(keys, dtype=np.uint64)
    return keys >> S32, keys & M32


def _simple(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Drop self-loops and repeats; keys in first-appearance order."""
    keep = u != v
    keys = pack(u[keep], v[keep])
    _, first = np.unique(keys, return_index=True)
    return keys[np.sort(first)]


def chung_lu(n: int, gamma: float, mean_degree: float, m: int | None,
             seed: int, max_degree: float | None = None) -> np.ndarray:
    """Chung-Lu style power-law graph by endpoint sampling.

    Vertex i gets weight (i+1)^(-1/(gamma-1)), scaled so the weights average
    ``mean_degree`` and optionally capped at ``max_degree``; each sampled edge
    draws both endpoints independently with probability proportional to the
    weights.  Samples are drawn until ``m`` distinct non-loop edges exist
    (m = n * mean_degree / 2 when None), then truncated to m in sample order.
    """
    rng = np.random.default_rng(seed)
    wts = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    wts *= mean_degree / wts.mean()
    if max_degree is not None:
        wts = np.minimum(wts, max_degree)
    cdf = np.cumsum(wts)
    cdf /= cdf[-1]
    if m is None:
        m = int(round(n * mean_degree / 2))
    have = np.zeros(0, dtype=np.uint64)
    want = m
    while True:
        k = int(want * 1.3) + 1024
        u = np.searchsorted(cdf, rng.random(k), side="right").astype(np.uint64)
        v = np.searchsorted(cdf, rng.random(k), side="right").astype(np.uint64)
        u = np.minimum(u, np.uint64(n - 1))
        v = np.minimum(v, np.uint64(n - 1))
        cat = np.concatenate([have, _simple(u, v)])
        _, first = np.unique(cat, return_index=True)
        have = cat[np.sort(first)]
        if have.size >= m:
            return have[:m]
        want = m - have.size


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float,
         seed: int) -> np.ndarray:
    """R-MAT (Chakrabarti et al.) with quadrant probabilities (a, b, c, d).

    edge_factor * 2^scale directed samples, symmetrised to (min, max),
    self-loops and repeats dropped.
    """
    rng = np.random.default_rng(seed)
    k = edge_factor << scale
    u = np.zeros(k, dtype=np.uint64)
    v = np.zeros(k, dtype=np.uint64)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        x = rng.random(k, dtype=np.float32)
        bit = np.uint64(1 << level)
        u |= np.where(x >= ab, bit, np.uint64(0))
        v |= np.where(((x >= a) & (x < ab)) | (x >= abc), bit, np.uint64(0))
    return _simple(u, v)


def finish(keys: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Relabel vertex ids by a random permutation and shuffle arrival order."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.uint64)
    u, v = unpack(keys)
    out = pack(perm[u.astype(np.int64)], perm[v.astype(np.int64)])
    return out[rng.permutation(out.size)]
