"""FP64 CPU oracle of the reactive two-component lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg import this package.  It shares no code
with the CUDA library and the product path never calls it.
"""
