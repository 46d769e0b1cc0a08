"""Kryging hot path on one GB300 (sm_103a): BTTB covariance matvec by circulant
embedding and hand-written FFT kernels, with the Krylov loops (stochastic
Lanczos quadrature, CG, GLS, kriging) that consume it.

The compute lives in the C-ABI library ``libkry.so`` (``include/kry.h``); the
Python binding in :mod:`paper_2012_13133_gb300.kry` marshals arguments only.
Importing this package loads nothing; import ``.kry`` to load the library.
"""
__version__ = "0.1.0"
