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


def chung_lu_device(n: int, gamma: float, mean_degree: float, m: int, seed: int,
                    max_degree: float | None = None, device: str = "cuda"):
    """Chung-Lu power-law stream of exactly m simple edges, drawn on the GPU.

    The recipe of ``graphs.chung_lu`` followed by ``graphs.finish``: vertex i
    has weight (i+1)^(-1/(gamma-1)) scaled to mean ``mean_degree`` and capped
    at ``max_degree``; each sample draws both endpoints independently with
    probability proportional to the weights (float64 uniforms into the
    weights' cumulative sum).  Self-loops and repeats are dropped, m of the
    distinct edges are kept in a uniformly random order, and vertex ids are
    relabelled by a random permutation.  Packed (min << 32) | max keys as an
    int64 tensor on `device`.  Drawn from torch's generator, so the edges
    differ from the numpy version; the same seed gives the same stream on
    the same GPU model and torch build.  Input generation only.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    wts = (torch.arange(n, dtype=torch.float64, device=device) + 1.0) ** (-1.0 / (gamma - 1.0))
    wts *= mean_degree / wts.mean()
    if max_degree is not None:
        wts.clamp_(max=max_degree)
    cdf = torch.cumsum(wts, 0)
    cdf /= cdf[-1].clone()
    del wts
    have = torch.zeros(0, dtype=torch.int64, device=device)
    want = m
    while True:
        k = int(want * 1.05) + 4096
        # both endpoints of k samples, drawn in chunks to bound the float64
        # temporaries
        parts = []
        for c0 in range(0, k, 1 << 28):
            c = min(1 << 28, k - c0)
            u = torch.searchsorted(cdf, torch.rand(c, dtype=torch.float64, generator=g,
                                                   device=device), right=True)
            v = torch.searchsorted(cdf, torch.rand(c, dtype=torch.float64, generator=g,
                                                   device=device), right=True)
            u.clamp_(max=n - 1)
            v.clamp_(max=n - 1)
            keep = u != v
            lo, hi = torch.minimum(u[keep], v[keep]), torch.maximum(u[keep], v[keep])
            del u, v, keep
            parts.append((lo << 32) | hi)
            del lo, hi
        have = torch.unique(torch.cat([have] + parts))
        del parts
        if have.numel() >= m:
            break
        want = m - have.numel()
    keys = have[torch.randperm(have.numel(), generator=g, device=device)[:m]]
    del have
    perm = torch.randperm(n, generator=g, device=device)
    pu, pv = perm[keys >> 32], perm[keys & 0xFFFFFFFF]
    del keys
    return (torch.minimum(pu, pv) << 32) | torch.maximum(pu, pv)
