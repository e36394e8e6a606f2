"""Plain FP64 CPU oracle for the block-Toeplitz Bayesian inversion hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, header, table or helper with the CUDA library; the two meet only in
the seeded input generator ``paper_2501_14911_gb300.synthetic``, which holds
no arithmetic of the method.

Every routine is the paper's definition written out in numpy float64, with a
library primitive (matmul, LAPACK Cholesky, triangular solve) as a step where
that is the plainest statement.  The FFT embedding that the CUDA path uses is
deliberately absent: the oracle computes the time-domain convolution sums the
FFT is supposed to reproduce exactly (Sec. 4, "FFT-based GPU-accelerated p2o and
p2q matvecs", and Eq. (2.4)-(2.5)).

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: simulation of the LTI recursion Eq. (2.2)-(2.3), the explicitly
assembled dense matrix Eq. (2.5), numpy.convolve, impulse responses, the
adjoint identity, the closed-form Gaussian posterior mean Eq. (2.12), the
Woodbury form Eq. (4.6)-(4.7), LAPACK-free Cholesky on small matrices, and
central finite differences of the quadratic loss.  No function here is
"parity unpinned".

Index conventions (0-based):
  blocks  [N_t][R][N_m]   block k = F_k = B A^k C (F_0 is the diagonal block)
  m       [..., N_t, N_m] parameter blocks m_0 .. m_{N_t-1}
  d       [..., N_t, R]   data blocks; d[t] depends on m[0..t]
  K       [(N_t R)][(N_t R)] with data index (t, i) -> t * R + i
"""

from .toeplitz import (
    p2o_apply,
    p2o_apply_adjoint,
    p2o_dense,
    p2o_apply_block,
    p2o_apply_adjoint_block,
    lti_blocks,
    lti_simulate,
)
from .prior import (
    se_covariance_1d,
    se_covariance,
    prior_blocks,
    prior_blocks_separable,
    prior_sample,
    elliptic_operator,
)
from .inversion import (
    assemble_K,
    assemble_K_columns,
    cholesky_lower,
    solve_K,
    map_point,
    map_point_woodbury_form,
    qoi_map,
    qoi_data_gram,
    d2q_map,
    qoi_posterior_covariance,
    prior_apply,
    posterior_cov_apply,
    posterior_variance_probe,
    map_point_with_prior_mean,
    qoi_time_steps,
    qoi_rows,
    loss,
    loss_gradient,
)

__all__ = [
    "p2o_apply", "p2o_apply_adjoint", "p2o_dense", "p2o_apply_block",
    "p2o_apply_adjoint_block", "lti_blocks", "lti_simulate",
    "se_covariance_1d", "se_covariance", "prior_blocks", "prior_blocks_separable", "prior_sample",
    "elliptic_operator",
    "assemble_K", "assemble_K_columns", "cholesky_lower", "solve_K",
    "map_point", "map_point_woodbury_form", "qoi_map", "qoi_data_gram", "d2q_map",
    "qoi_posterior_covariance", "prior_apply", "posterior_cov_apply", "posterior_variance_probe", "map_point_with_prior_mean",
    "qoi_time_steps", "qoi_rows", "loss", "loss_gradient",
]
