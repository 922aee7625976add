"""GB300 (sm_103a) setup path of the chiral rank-k multigrid preconditioner
for Wilson fermions (arXiv:2502.03091).

The compute path is the CUDA library libmg.so behind the C ABI in
include/mg.h; ``paper_2502_03091_gb300.mg`` is its ctypes binding.  Importing
this package does not load the library; the first ABI call does, and raises
if the library has not been built (``python -m paper_2502_03091_gb300.build``).
"""
from . import mg  # noqa: F401

__all__ = ["mg"]
