"""GB300-native hybrid lattice-Boltzmann Bloch-Torrey sweep (arXiv 1907.00908).

``lbmbt`` is the ctypes binding of the C-ABI library ``liblbmbt.so`` (CUDA,
sm_103a); ``synth`` makes seeded input geometries.  Importing the package does
not load the CUDA library; ``lbmbt.lib()`` does, and raises if it is missing.
"""
