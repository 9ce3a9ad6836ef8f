"""CPU oracle for bulk neighborhood-sampling triangle counting.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` use it.  It shares no code with the CUDA path: its Philox, its
bounded draw, its sorts and its searches are written here from the published
definitions, in plain Python and numpy.

Modules (each cites the passage of Tangwongsan, Pavan and Tirthapura,
"Parallel Triangle Counting in Massive Streaming Graphs", that it follows):

* ``philox``     -- Philox4x32-10 (Salmon et al., SC'11), scalar and numpy.
* ``draws``      -- Lemire's nearly-divisionless bounded draw and the fixed
                    draw conventions (which Philox words each step consumes).
* ``nbsi``       -- the batched update ``bulkUpdateAll`` (Sec. 4), written
                    per estimator with an injectable draw source (scalar).
* ``nbsi_bulk``  -- the same update written with the paper's bulk primitives
                    (map / sort / scan-with-resets / multisearch, Sec. 3.2,
                    Sec. 4) over numpy arrays, for the large configurations.
* ``sequential`` -- the edge-at-a-time neighborhood-sampling estimator
                    (batch size one, Sec. 4.2), an independent formulation.
* ``enumerate``  -- exact (rational) distributions of the estimator state by
                    exhaustive enumeration of every draw outcome.
* ``exact``      -- exact triangle counts and per-triangle C(t*) (Sec. 2).
* ``estimate``   -- the 128-bit estimate of Lemma 3.1 / Eq. for tau_hat, and
                    median-of-means (Sec. 3.1).

Every function is pinned by ``tests/test_oracle_*.py`` against facts that do
not come from the oracle itself (the worked example of Figs. 1-3, exhaustive
probabilities from the Claim of Sec. 3.1, closed forms, published Philox
known-answer vectors); see each module's header for its pins.
"""
