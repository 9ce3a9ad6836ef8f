"""R-MAT edge streams sampled on the GPU (torch), for workloads too large to
generate in numpy within a benchmark run (the serving mix draws from R-MAT
graphs of scale 14 to 22, up to 67M samples each).

Same recipe as ``graphs.rmat`` followed by ``graphs.finish`` -- quadrant
probabilities (a, b, c, 1-a-b-c) per level, symmetrised to (min, max),
self-loops and repeats dropped, vertex ids relabelled by a random
permutation, arrival order shuffled -- but drawn from torch's generator, so
the edges differ from the numpy version for the same seed.  Input generation
only: nothing of the triangle-counting method is computed here.
"""
from __future__ import annotations


def rmat_device(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
                device: str = "cuda"):
    """Packed simple edges (min << 32) | max as an int64 tensor on `device`,
    in random arrival order."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    k = edge_factor << scale
    u = torch.zeros(k, dtype=torch.int64, device=device)
    v = torch.zeros(k, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        x = torch.rand(k, generator=g, device=device)
        u |= (x >= ab).to(torch.int64) << level
        v |= (((x >= a) & (x < ab)) | (x >= abc)).to(torch.int64) << level
        del x
    lo, hi = torch.minimum(u, v), torch.maximum(u, v)
    del u, v
    keep = lo != hi
    keys = torch.unique((lo[keep] << 32) | hi[keep])
    del lo, hi, keep
    perm = torch.randperm(1 << scale, generator=g, device=device)
    pu, pv = perm[keys >> 32], perm[keys & 0xFFFFFFFF]
    keys = (torch.minimum(pu, pv) << 32) | torch.maximum(pu, pv)
    del pu, pv
    return keys[torch.randperm(keys.numel(), generator=g, device=device)]
