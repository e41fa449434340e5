"""GB300-native projected EM for 2D super-resolution multi-reference alignment.

The compute path lives in the CUDA library ``libsrmra.so`` (C ABI declared in
``include/srmra.h``); :mod:`paper_2204_04754_gb300.srmra` is a thin ctypes binding
with the same entry-point names.  :mod:`paper_2204_04754_gb300.synth` generates the
seeded synthetic inputs.  Importing this package does not load the CUDA library;
the binding loads it on first use and raises if it is missing.
"""

__all__ = ["synth", "srmra", "build"]
