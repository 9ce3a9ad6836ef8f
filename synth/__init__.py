"""Seeded synthetic edge streams shaped like the paper's social graphs.

This package holds the input generators only -- none of the triangle-counting
arithmetic -- so that both the CUDA path's tests/benchmarks and the CPU
oracle can consume the same inputs.  Every stream is a uint64 array of packed
edges (min << 32) | max in arrival order: simple (no self-loops, no repeats),
vertex ids randomly relabelled, arrival order a seeded uniform permutation.

The paper's datasets (SNAP Amazon, DBLP, LiveJournal, Orkut, Friendster, a
Twitter graph, a 167 GB power-law graph; Table 1) are not available; these
generators stand in for them with the same shape: power-law degrees,
m from 1e4 to 1e9 edges.
"""
from .graphs import chung_lu, rmat, finish, pack, unpack  # noqa: F401
from .workloads import (WORKLOADS, LARGE_EDGES, tiny_chung_lu, rmat20_single, large_prefix,  # noqa: F401
                        large_stream_device, batches, multi_streams,
                        multi_streams_device)
