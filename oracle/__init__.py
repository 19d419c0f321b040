"""FP64 CPU oracle of the forced EVD lattice Boltzmann step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does.
"""
