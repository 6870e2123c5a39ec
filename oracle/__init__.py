"""Oracle for the learnable multigrid: test infrastructure only.

Only tests, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from .lmg import (Hierarchy, Level, Params, build_hierarchy, cheb_conv, conv, fgmres,  # noqa: F401
                  fmg, lap_hat, lmg, loss_gradient_complex_step, loss_gradient_fd, relres, residual,
                  smooth, solve_refinement, solve_vcycles, unrolled_loss, vcycle)
