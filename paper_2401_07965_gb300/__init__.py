"""GB300-native population annealing (arXiv:2401.07965, Sec. 2-3).

The hot path -- checkerboard Metropolis sweeps of bit-packed Ising / EA +-J
replicas, reweighting and Q, the five copy-count rules and the replica copy --
runs in the CUDA kernels of lib/libpa.so behind the C ABI of include/pa.h.
`paper_2401_07965_gb300.pa` is the thin Python binding of that ABI; importing
it loads libpa.so and fails if the library is not built.
"""
