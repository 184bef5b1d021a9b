"""GB300-native FFT chemo-mechanical fracture solver (arXiv 2411.16583).

The method runs in the CUDA library built from ``csrc/`` (see ``build.py``) behind the
C ABI of ``include/fg.h``; ``binding`` marshals arguments to it and ``synth`` generates
seeded workloads.  Importing the package does not load the library.
"""
__all__ = ["binding", "synth", "build"]
