"""FP64 CPU oracle for the multi-scale low rank decomposition (Ong & Lustig).

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously correct
restatement of what the GPU path computes, written in float64 NumPy straight
from the paper (Sec. 3 eq:cvx, Sec. 7 eq:svt / eq:bsvt / eq:admm, Sec. 9
random cycle spinning, Sec. 10.4 masked X-update).  Only the tests, the
smoke check and the benchmark's CPU-baseline / reference arm may import it;
the product path (the CUDA library and its Python binding) never does, and
shares no code with it.

Parity status per function (what pins each one is listed in the tests):
  shift_table          pinned (published splitmix64 output, range/uniformity)
  lambda_default       pinned (closed forms of eq:lambda at the 1x1 / MxN ends)
  svt / block_svt      pinned (closed-form singular values, brute-force prox
                        optimality on 2x2 / 3x3, textbook 1x1 and 1xN cases)
  admm                 pinned with shifts off (KKT / duality certificate of
                        the convex program, exact recovery, homogeneity);
                        with random cycle spinning: parity unpinned against
                        the paper (it prints no numbers), pinned only by the
                        per-iteration invariants sum_i X_i = Y and U' = A - Z'.
  blocks3d / block_svt_3d   pinned (inverse of its adjoint, reduction to the
                        2-D partition when a block spans whole frame rows,
                        brute force by explicit pixel indices)
  spin_set /           pinned (exact translation equivariance over the full
  block_svt_spun        set, identity at tau = 0, brute force by explicit
                        block windows, single-shift special case; the
                        averaged ADMM is translation equivariant)
"""

from .msllr_oracle import (  # noqa: F401
    splitmix64,
    shift_table,
    lambda_default,
    lambda_area,
    shift,
    unshift,
    svt,
    soft_threshold,
    block_svt,
    spin_set,
    block_svt_spun,
    blocks3d,
    unblocks3d,
    shift3d,
    block_svt_3d,
    block_nuclear_norm,
    block_dual_norm,
    consensus_residual,
    x_update,
    admm,
    admm_step,
    relerr,
)
