"""Piece-wise-constant-tested isogeometric analysis on GB300 (sm_103a).

The compute path is the C-ABI library ``lib/libigapw.so`` (hand-written CUDA
kernels, see ``include/igapw.h``).  ``igapw`` is a thin ctypes binding with the
same call names plus a small ``Context`` convenience wrapper that allocates
torch tensors of the right shape; torch supplies device memory and streams
only.  Importing this package does not load the library; the first call does,
and fails loudly if it has not been built.
"""
__all__ = ['igapw', 'workloads']
