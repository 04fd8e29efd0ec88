"""GB300-native velocity-gauge real-time TDDFTB density-matrix propagation.

The compute path is the C-ABI library ``libvgtb.so`` (CUDA kernels for
sm_103a) built from ``csrc/``; ``vgtb`` is its thin ctypes binding and
``inputs`` builds seeded synthetic systems.  Importing the package does not
load the library; ``vgtb.load()`` does, and fails loudly when it is missing.
"""
