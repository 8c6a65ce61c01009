"""GB300 (sm_103a) encrypted 1:N face matching: CKKS plaintext-template x
encrypted-query BSGS product with hoisted baby steps and pre-rotated
diagonals, Chebyshev threshold and membership slot sum (arXiv 2604.00546).

The computation lives in libfr.so (C ABI: include/fr.h); ``fr`` is its
Python binding and ``workloads`` the seeded synthetic inputs.
"""
from . import build  # noqa: F401
