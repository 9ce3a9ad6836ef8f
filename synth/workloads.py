"""The named workloads: graph, estimator count r, batch size w, seeds.

* ``tiny``    Chung-Lu, exponent 2.3, n = 4096, m = 32768 (mean degree 16),
              r = 1024, w = 4096, Philox seed 1.
* ``rmat20``  R-MAT scale 20, edge factor 16, (a, b, c, d) =
              (0.57, 0.19, 0.19, 0.05), symmetrised and deduplicated
              (about 15M edges), r = 2^20, w = 2^22.
* ``large``   Chung-Lu, exponent 2.1, n = 2^25, maximum expected degree 3e5,
              r = 2^24, w = 2^24 (about 1.2e9 edges in the full stream).
"""
from __future__ import annotations

import numpy as np

from .graphs import chung_lu, finish, rmat

WORKLOADS = {
    "tiny": dict(graph="chung-lu gamma=2.3 n=4096 m=32768", n=4096, r=1024,
                 w=4096, seed=1, vertex_bits=12),
    "rmat20": dict(graph="r-mat scale=20 ef=16 (0.57,0.19,0.19,0.05)",
                   n=1 << 20, r=1 << 20, w=1 << 22, seed=1, vertex_bits=20),
    "large": dict(graph="chung-lu gamma=2.1 n=2^25 dmax=3e5", n=1 << 25,
                  r=1 << 24, w=1 << 24, seed=1, vertex_bits=25),
}


def tiny_chung_lu(gen_seed: int = 1) -> np.ndarray:
    n = 4096
    keys = chung_lu(n, 2.3, 16.0, 32768, seed=gen_seed)
    return finish(keys, n, seed=gen_seed + 1000)


def rmat20_single(gen_seed: int = 1, scale: int = 20) -> np.ndarray:
    keys = rmat(scale, 16, 0.57, 0.19, 0.19, seed=gen_seed)
    return finish(keys, 1 << scale, seed=gen_seed + 1000)


def large_prefix(n_batches: int = 2, gen_seed: int = 1) -> np.ndarray:
    """The first n_batches * 2^24 edges of the ``large`` stream.

    Chung-Lu, exponent 2.1, n = 2^25, expected degrees scaled to the full
    stream's mean (2 * 1.2e9 / 2^25, about 71.5) and capped at 3e5.  Endpoint
    sampling draws every edge independently, so the first k distinct samples
    (relabelled, in random order) are a prefix of a random-order stream of
    the full graph; only that prefix is generated.
    """
    n = 1 << 25
    mean_degree = 2 * 1.2e9 / n
    keys = chung_lu(n, 2.1, mean_degree, n_batches << 24, seed=gen_seed, max_degree=3e5)
    return finish(keys, n, seed=gen_seed + 1000)


# Edges of the whole ``large`` stream (about 1.2e9, 71.5 batches of 2^24).
LARGE_EDGES = 1_200_000_000


def large_stream_device(m: int = LARGE_EDGES, gen_seed: int = 1, device: str = "cuda"):
    """The ``large`` stream drawn on the GPU: Chung-Lu, exponent 2.1,
    n = 2^25, expected degrees with mean 2 * 1.2e9 / 2^25 (about 71.5)
    capped at 3e5, m distinct edges in random order (int64 tensor of packed
    keys on `device`).  m defaults to the whole stream, so that every batch a
    run folds in is a new one (no batch is replayed); a smaller m is a
    shorter stream from the same degree weights, not a prefix of it."""
    from .device import chung_lu_device
    n = 1 << 25
    return chung_lu_device(n, 2.1, 2 * LARGE_EDGES / n, m, seed=gen_seed, max_degree=3e5,
                           device=device)


def batches(keys: np.ndarray, w: int):
    """Split a stream into consecutive batches of w edges (last may be short)."""
    return [keys[i:i + w] for i in range(0, keys.size, w)]


def multi_streams(S: int = 512, per_stream_edges: int = 32768, seed: int = 1,
                  m_range=(1e4, 1e7), r_range=(2 ** 10, 2 ** 16), gamma_range=(2.1, 2.5),
                  mean_degree: float = 16.0):
    """S independent Chung-Lu streams for the batched multi-stream workload.

    Stream s draws m_s log-uniform in m_range (its full length), r_s
    log-uniform in r_range, exponent uniform in gamma_range, n_s = 2 m_s /
    mean_degree vertices; only the first min(m_s, per_stream_edges) edges of
    each stream are generated (the first distinct samples of its endpoint-
    sampling process, relabelled and put in random order), which is all a
    bounded number of rounds consumes.  Returns (streams, r, n).
    """
    rng = np.random.default_rng(seed)
    lm = rng.uniform(np.log(m_range[0]), np.log(m_range[1]), size=S)
    lr = rng.uniform(np.log(r_range[0]), np.log(r_range[1]), size=S)
    gam = rng.uniform(gamma_range[0], gamma_range[1], size=S)
    streams, rs, ns = [], [], []
    for s in range(S):
        m = int(np.exp(lm[s]))
        n = max(64, int(2 * m / mean_degree))
        k = min(m, per_stream_edges)
        keys = chung_lu(n, float(gam[s]), 2.0 * m / n, k, seed=seed * 100_003 + s)
        streams.append(finish(keys, n, seed=seed * 100_003 + s + 50_000))
        rs.append(int(np.exp(lr[s])))
        ns.append(n)
    return streams, np.array(rs, dtype=np.uint64), np.array(ns, dtype=np.int64)


def multi_streams_device(S: int = 512, seed: int = 1, m_range=(1e4, 1e7),
                         r_range=(2 ** 10, 2 ** 16), gamma_range=(2.1, 2.5),
                         mean_degree: float = 16.0, device: str = "cuda"):
    """S independent Chung-Lu streams at their full lengths, drawn on the GPU.

    Stream s has m_s edges, m_s log-uniform in m_range; r_s estimators,
    log-uniform in r_range; exponent uniform in gamma_range; n_s =
    max(64, 2 m_s / mean_degree) vertices.  Returns (streams, r, n): a list
    of int64 device tensors of packed edges in arrival order, and numpy
    arrays of r_s and n_s.
    """
    from .device import chung_lu_device
    rng = np.random.default_rng(seed)
    lm = rng.uniform(np.log(m_range[0]), np.log(m_range[1]), size=S)
    lr = rng.uniform(np.log(r_range[0]), np.log(r_range[1]), size=S)
    gam = rng.uniform(gamma_range[0], gamma_range[1], size=S)
    streams, rs, ns = [], [], []
    for s in range(S):
        m = int(np.exp(lm[s]))
        n = max(64, int(2 * m / mean_degree))
        streams.append(chung_lu_device(n, float(gam[s]), 2.0 * m / n, m,
                                       seed=seed * 100_003 + s, device=device))
        rs.append(int(np.exp(lr[s])))
        ns.append(n)
    return streams, np.array(rs, dtype=np.uint64), np.array(ns, dtype=np.int64)
