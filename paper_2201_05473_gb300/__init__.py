"""GB300-native lattice-Boltzmann plasma-wakefield step (arXiv:2201.05473).

The compute path is the C-ABI library ``libpwfa_lbm.so`` (hand-written CUDA for
sm_103a) declared in ``include/pwfa_lbm.h``; ``paper_2201_05473_gb300.lbm``
binds it with ctypes. Importing this package does not load the library, so the
input generators in ``workloads`` can be used on a machine without a GPU.
"""

__all__ = ["workloads"]
