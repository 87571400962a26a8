"""GB300 library for many-particle continuous-time quantum walks on noisy lattices.

Implements the hot path of Piccinini et al., arXiv:1612.00746: the truncated
Taylor series of the evolution operator (Sec. 2.3, Algorithm 3) and RK4
(Sec. 2.2, Algorithm 2) on stochastic tight-binding Hamiltonians (Eq. (Hij)),
with ensemble-averaged site occupations.  The compute path is the CUDA
library libctqw.so (sm_103a); ``ctqw`` is its ctypes binding.
"""
from . import ctqw  # noqa: F401
