"""Oracle for the learnable multigrid: test infrastructure only.

Only tests, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from .lmg import (Hierarchy, Level, Params, Params2, build_hierarchy, cheb_conv,  # noqa: F401
                  cheb_gradient_complex_step, cheb_gradient_fd,
                  complex_vec, conv, conv2, fcg, features, fgmres, fgmres2, fmg, fmg2,
                  lap_hat,
                  lmg, lmg2, real_vec,
                  loss_gradient_complex_step, smooth2, vcycle2, loss_gradient_fd, relres, residual,
                  smooth, solve_refinement, solve_vcycles, unrolled_loss, vcycle)
