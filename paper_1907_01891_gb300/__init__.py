"""GB300-native QR-based CT reconstruction (Chillaron et al., 1907.01891).

The compute lives in the CUDA library ``libctqr.so`` behind the C ABI of
``include/ctqr.h``; ``paper_1907_01891_gb300.ctqr`` is the thin ctypes binding.
Importing the package itself loads nothing.
"""
