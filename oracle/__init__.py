"""CPU oracle for the AA-QAOA hot path: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything from this package. It is an independent FP64
statement of what the CUDA library computes and shares no code with it.

Modules:
  oracle        -- ctypes front end of the plain C statevector oracle
  closed_form   -- published p = 1 edge expectation (any graph, any n)
  symmetric     -- Dicke-subspace oracle for K_n and stars (any n, any p)
  lightcone     -- per-edge light-cone evaluation with the full oracle
  automorphisms -- brute-force automorphism groups for small graphs
"""
