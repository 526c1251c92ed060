"""FP64 CPU oracle for the chance-constrained GP-MPPI rollout.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the paper defines (Trivedi et al., "Data-Driven Sampling
Based Stochastic MPC for Skid-Steer Mobile Robot Navigation"): Eq. 1-3 and
Eq. 10 for the motion model, Eq. 11-16 for costs and chance constraints,
Alg. 1 Step 1 / Step 2 for the MPPI iteration, and Eq. 3-4 (Step 3) for the
terrain ensemble and its weights.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA path; both take their inputs
from the ``scenarios`` module, which holds no arithmetic of the method.

Every floating-point step runs in float64.  Library primitives (a Cholesky,
a triangular solve, an eigen-solve of a 2x2) serve as steps; nothing is
blocked, fused or reordered beyond the definitions.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  philox4x32_10 / normals ... pinned (cuRAND host generator, moments)
  gp_fit / gp_predict ...... pinned (N=1 closed form, far field, sklearn)
  dynamics / covariance .... pinned (straight-line, arc, matrix-power forms)
  costs / tightening ....... pinned (quantile closed forms, scipy, eigvalsh,
                              hand-computable straight-path cases)
  weights / update ......... pinned (sum to one, temperature limits, K=1)
  smoothed objective / gradient ... pinned (Richardson agreement, the
                              straight-line analytic gradient, sigmoid ->
                              indicator as the slope grows)
  terrain ensemble (Eq. 3) . pinned (M = 1 is the single GP, one-hot weights
                              select a terrain, identical terrains give the
                              mean times sum w and the variance times sum w^2)
  goal terms (Eq. 12) ...... pinned (hand-computable straight-line cases)
  terrain weights (Eq. 4) .. pinned (exact recovery, the equality-constrained
                              least-squares closed form, the large-gamma limit,
                              brute force over a fine simplex grid)
  nominal tightening mode .. parity unpinned beyond the zero-noise identity
                              with the per-sample mode (the placement of
                              Alg. 1 Step 2 is a reading, not a definition)
"""

from .philox import philox4x32_10, uniforms_from_words, box_muller, control_noise  # noqa: F401
from .quantiles import chi2_2_quantile, normal_quantile  # noqa: F401
from .gp import se_ard, gp_fit, gp_predict, Ensemble, gp_predict_ensemble, predict, fit_scenario  # noqa: F401
from .mppi import (  # noqa: F401
    nominal_step, jacobian, covariance_step, lane_distance, lambda_max_2x2,
    stage_cost, rollout, mppi_weights, mppi_update, mppi_step, nominal_tightening,
    Controller,
)
from .gradient import objective, fd_gradient, with_lengthscale  # noqa: F401
from .terrain import terrain_weights, terrain_objective  # noqa: F401
