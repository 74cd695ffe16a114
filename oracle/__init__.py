"""CPU oracle for Scylla's hot path (arXiv 2307.03466) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the CUDA path computes: the PDHG solve of
the LP relaxation (Algorithm 1, Sections 2.1-2.2), fix-and-propagate (Section 2.3),
cycle handling (Section 2.3) and the objective update (Section 2.4, Algorithm 1).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call or run anything in this package.  It shares no code
with the CUDA path and imports nothing from it.
"""
