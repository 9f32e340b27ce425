"""GB300-native compact gas-kinetic scheme with GENO reconstruction.

The compute path lives in ``csrc/`` (sm_103a CUDA kernels behind a C-ABI
library, ``libgenogks.so``); :mod:`.binding` is the thin ctypes layer over it.
:mod:`.inputs` builds seeded synthetic initial data.
"""
