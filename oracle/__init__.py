"""FP64 CPU oracle of the compressible Navier-Stokes right-hand side and RK3 update.

Test infrastructure: only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library.
"""
