"""GB300-native compressible Navier-Stokes right-hand side and Wray RK3 update (STREAmS method,
arXiv 2004.02276), as a C-ABI CUDA library for sm_103a with a thin Python binding.

``inputs`` holds the seeded workload generators; ``binding`` loads ``libstrm.so`` (built by
``__graft_entry__.build()``) and raises if it is missing.
"""
