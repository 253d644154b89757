"""GB300-native cue-field diffusion and growth-cone steering (sm_103a).

The compute path lives in ``libcue.so`` (hand-written CUDA behind a C ABI,
declared in ``include/cue.h``); :mod:`paper_1405_3331_gb300.cue` is the thin
Python binding over it.  Importing the package itself loads nothing.
"""
