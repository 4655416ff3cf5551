"""GB300-native ASIFT-view + ORB + Hamming matching (arXiv 2503.03479 hot path).

The compute path is the CUDA library ``libasift.so`` (built from ``csrc/`` for
sm_103a); ``asift`` is its thin ctypes binding.  ``synth`` holds the seeded
synthetic input generators.
"""
