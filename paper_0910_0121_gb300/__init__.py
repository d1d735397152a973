"""GB300-native periodic short-range tree force of GreeM (Ishiyama, Fukushige & Makino 2009).

The compute path is ``libgreem.so`` (hand-written CUDA for sm_103a behind a C ABI,
``include/greem.h``); :mod:`paper_0910_0121_gb300.greem` is a thin ctypes binding that
only marshals arguments.  :mod:`paper_0910_0121_gb300.synth` draws the seeded synthetic
particle sets.
"""
__all__ = ["greem", "synth"]
