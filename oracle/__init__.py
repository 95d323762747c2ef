"""FP64 CPU oracle of the finite-difference wave propagator (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA library never does.
"""
