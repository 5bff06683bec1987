"""FP64 CPU oracle of the Gaussian lattice Boltzmann method (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package. It shares no code with the CUDA library.
"""
