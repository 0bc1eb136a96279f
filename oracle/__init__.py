"""Plain, slow FP64 CPU oracle for the relativistic CCSD / FS-CCSD(0h1p) hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its Python binding) never calls it and shares no code with it;
the only module both sides use is the seeded input generator
``paper_2004_03682_gb300.synthetic``, which holds random draws and no method
arithmetic.

Every function here is a direct transcription of a definition (dense complex128
numpy arrays, einsum for each term), with no blocking, packing or fusion, so that
it can be read against the equations it cites.
"""
