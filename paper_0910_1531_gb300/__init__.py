"""GB300-native (sm_103a) FFT/Picard classical-DFT hot path for charged hard spheres.

The compute path is the C-ABI library ``libgb300dft.so`` built from ``csrc/``;
``binding`` marshals arguments to it.  ``workloads`` builds seeded synthetic
inputs.  Importing this package loads nothing; the library is loaded on first
use and a missing or unloadable library raises an error (there is no CPU
fallback).
"""
