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


def batches(keys: np.ndarray, w: int):
    """Split a stream into consecutive batches of w edges (last may be short)."""
    return [keys[i:i + w] for i in range(0, keys.size, w)]
