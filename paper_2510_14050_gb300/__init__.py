"""GB300-native anonymized network sensing: traffic matrices (DCSR) and the
Graph Challenge network quantities from windows of (src, dst) packet pairs.

Submodules are imported on demand so that the generator (``synth``) can be
used without loading the CUDA library:

* ``paper_2510_14050_gb300.ans``   -- ctypes binding of ``include/ans.h``
* ``paper_2510_14050_gb300.synth`` -- seeded synthetic windows
"""
__all__ = ["ans", "synth", "buildlib"]
