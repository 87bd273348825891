"""GB300 (sm_103a) implementation of the data-parallel hot path of the
four-dimensional overlapping domain-decomposition factorization of the
Wilson-Dirac fermion determinant (Saccardi & Giusti, Lattice 2022).

The compute lives in the CUDA library ``libdd4d.so`` (C-ABI declared in
``include/dd4d.h``); :mod:`paper_2211_06902_gb300.dd4d` is its thin ctypes
binding and :mod:`paper_2211_06902_gb300.synth` the seeded input generators.
"""
