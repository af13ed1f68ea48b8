"""Piece-wise-constant-tested isogeometric analysis on GB300 (sm_103a).

The compute path is the C-ABI library ``lib/libigapw.so`` (hand-written CUDA
kernels, see ``include/igapw.h``). ``igapw`` is a thin ctypes binding with the
same call names plus two convenience wrappers that allocate torch tensors of
the right shape and check the ones they are given: ``Context`` (one problem:
tables, operator action, source RHS, Kronecker solve, explicit steps, 2D/3D
Poisson with Dirichlet or mixed boundary conditions) and ``Batch`` (many
uneven 2D Poisson instances solved stage by stage in shared launches).
``serve`` is a continuous-batching request server on top of contexts;
``workloads`` holds the seeded input generators; ``profile_cases`` small runs
for profiler captures. Torch supplies device memory and streams only.
Importing this package does not load the library; the first call does, and
fails loudly if it has not been built.
"""
__all__ = ['igapw', 'workloads', 'serve', 'profile_cases']
