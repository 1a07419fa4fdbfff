"""GB300 (sm_103a) implementation of the TRSTMI stochastic trust-region
coherence search (arXiv 2207.06374) behind a C ABI (include/trstmi.h).

`paper_2207_06374_gb300.trstmi` is the ctypes binding of libtrstmi.so;
`paper_2207_06374_gb300.build` compiles it in-tree.
"""
