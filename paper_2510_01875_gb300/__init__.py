"""GB300-native LR-TDDFT response path: pair densities, Adler-Wiser chi0, Dyson, S(q,w),
F(q,tau) and the constraints-based attenuation of narrow-band fluctuations.

The compute lives in the CUDA library built from csrc/ (liblrtddft.so, C ABI declared in
include/lrtddft.h); `binding` marshals arguments to it.  Importing this package does not
load the library; `paper_2510_01875_gb300.binding.load()` does, and fails loudly when it
is missing.
"""
