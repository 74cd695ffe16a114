"""GB300 (sm_103a) implementation of the PDHG hot path of the Scylla MIP heuristic
(arXiv 2307.03466).  ``scylla`` is the binding of the C ABI in include/scylla.h,
``build`` compiles the native library, ``instances`` draws seeded test MIPs."""
