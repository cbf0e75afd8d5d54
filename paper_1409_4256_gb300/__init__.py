"""GB300-native EMC (Expand-Maximize-Compress) hot path.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through the ctypes binding in ``emc.py`` (imported lazily so that the seeded
input generator ``synth`` can be used without the library).
"""
