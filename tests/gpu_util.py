"""Helpers shared by the GPU tests (device transfer, state comparison)."""
import numpy as np


def to_device(keys):
    import torch
    return torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)).cuda()


def assert_state_equal(got, exp, where=""):
    names = ("f1", "f2", "chi", "flags")
    for g, e, name in zip(got, exp, names):
        g = np.asarray(g, dtype=np.uint64)
        e = np.asarray(e, dtype=np.uint64)
        if not np.array_equal(g, e):
            bad = np.flatnonzero(g != e)
            raise AssertionError(f"{where} {name}: {bad.size} estimators differ, first {bad[:5]} "
                                 f"gpu={g[bad[:5]]} oracle={e[bad[:5]]}")
