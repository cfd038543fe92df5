"""GB300-native BinarySkyHough number count (Covas & Sintes, arXiv:1904.04873).

The hot path (peakgram, weights, FP64 track tables, number count with a
fused per-patch toplist, stage-2 power sum) runs in hand-written CUDA for
sm_103a behind the C ABI declared in ``include/bsh.h``.  ``bsh`` is the thin
ctypes binding to that library; ``synth`` makes seeded synthetic inputs.
Importing the package does not load the CUDA library.
"""
__all__ = ["synth", "bsh"]
