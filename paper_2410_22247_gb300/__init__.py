"""GB300-native AA-QAOA hot path: statevector QAOA for MaxCut with the full
H_C or the orbit-reduced H_red observable, energy and adjoint gradient, in
hand-written sm_103a CUDA behind a small C ABI (``include/aaqaoa.h``)."""
