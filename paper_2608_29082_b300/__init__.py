"""B300 learnable graph-convolution geometric multigrid.

The V-cycle of "A Learnable Multigrid Framework via Graph Convolutions"
(Algorithm 2) runs in hand-written CUDA kernels for sm_103a inside libmg.so
(C ABI in include/mg.h).  This package is its thin Python binding.
"""
from ._lib import MGError, lib  # noqa: F401
from .hierarchy import Hierarchy  # noqa: F401
from .solver import LMGParams, SolveInfo, Solver  # noqa: F401
