"""GB300-native free-surface lattice Boltzmann (FSLBM) time step.

The compute path is the CUDA library ``libfslbm`` (hand-written sm_103a
kernels behind a C ABI, declared in ``include/fslbm.h``); ``fslbm`` is its thin
ctypes binding and ``scenarios`` holds the seeded synthetic initial states.
"""
