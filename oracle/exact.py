"""Exact triangle counts and per-triangle quantities (oracle helpers).

Sec. 2 defines tau(G), the set T(G) of triangles and, for a triangle t*,
C(t*) = |Gamma(f)| where f is the first edge of t* in stream order.  These
are the quantities the Claim and Lemma 3.1 of Sec. 3.1 are stated in, and the
exact count against which the estimate's relative error is reported.

* ``triangles`` / ``C_values`` / ``gamma`` -- brute force, tiny graphs.
* ``count_dense`` -- trace(A^3)/6 with a dense matrix product (n <= ~8k).
* ``count`` -- the forward algorithm in C (``exact_count.c``), any size.

Pins: tests/test_oracle_exact.py (closed forms for K_n, K_{a,b}, wheels;
the three counters against each other on random graphs).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libexact_count.so")
_lib = None


def build() -> str:
    """Compile the C forward-algorithm counter (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "exact_count.c")
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_count_triangles.restype = ctypes.c_uint64
        lib.oracle_count_triangles.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                               ctypes.c_uint32]
        _lib = lib
    return _lib


def count(keys: np.ndarray, n: int | None = None) -> int:
    """tau(G) for packed keys (u<<32)|v, u < v, by the forward algorithm."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    if keys.size == 0:
        return 0
    if n is None:
        n = int((keys & np.uint64(0xFFFFFFFF)).max()) + 1
    t = _load().oracle_count_triangles(keys.ctypes.data, keys.size, n)
    if t == (1 << 64) - 1:
        raise MemoryError("exact triangle count ran out of memory")
    return int(t)


def count_dense(keys: np.ndarray, n: int) -> int:
    """tau(G) = trace(A^3) / 6 with a dense adjacency matrix."""
    A = np.zeros((n, n), dtype=np.float64)
    u = (keys >> np.uint64(32)).astype(np.int64)
    v = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    A[u, v] = 1.0
    A[v, u] = 1.0
    t = np.einsum("ij,ji->", A @ A, A)
    return int(round(t)) // 6


def triangles(edges):
    """All triangles of a tiny graph as frozensets of three edges."""
    es = {tuple(sorted(e)) for e in edges}
    verts = sorted({x for e in es for x in e})
    out = []
    for a, b, c in itertools.combinations(verts, 3):
        if (a, b) in es and (a, c) in es and (b, c) in es:
            out.append(frozenset({(a, b), (a, c), (b, c)}))
    return out


def gamma(edges, e):
    """Gamma(e): edges sharing a vertex with e that arrive after it (Sec. 2)."""
    order = [tuple(x) for x in edges]
    i = order.index(tuple(e))
    return [f for f in order[i + 1:] if len(set(f) & set(e)) == 1]


def C_values(edges):
    """C(t*) = |Gamma(first edge of t*)| for every triangle (Sec. 2)."""
    order = [tuple(x) for x in edges]
    pos = {e: i for i, e in enumerate(order)}
    out = []
    for t in triangles(order):
        first = min(t, key=lambda e: pos[e])
        out.append(len(gamma(order, first)))
    return out
