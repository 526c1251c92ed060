"""Chance-constrained GP-MPPI iteration in FP64 (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (the paper leaves these open):
  * f_v, f_omega (Eq. 1-2) are first-order velocity lags with time constants
    tau_v, tau_w; positions and heading integrate v(k), theta(k), omega(k) by
    explicit Euler (Sec. III-A says positions are integrated velocities).
  * Eq. 10's Jacobian is that of the nominal f only (GP mean not
    differentiated), evaluated at the pre-step mean and the clamped control.
  * GP variance is that of the latent function; one terrain (M = 1, w = 1)
    in Eq. 3, so C is diag(var_v, var_omega) and trace(C) = var_v + var_omega.
  * GP query at step k is (mu_v(k), mu_omega(k), u~_v(k), u~_omega(k)), where
    u~ is the perturbed control clamped to [u_min, u_max] (Eq. 8).
  * Stage k = 0..T-1 is scored on the state after the k-th update, mu(k+1)
    and Sigma(k+1), with GP covariance C(k) of that update and discount 0.9^k.
  * Deviation d = e / r with e the distance to the centre polyline and r the
    nominal half-width; the lane indicator of Eq. 11 fires when e > r_bar
    (Eq. 14); the collision indicator of Eq. 12 fires when min_j d_bar_j <= 0
    (Eq. 16); indicator weights are alpha_3 * P_lane and beta_1 * P_coll.
  * Speed term: alpha_4 * (v_desired - mu_v)^2 (squared so that both signs
    of deviation are penalised).
  * Slip (alpha_2) is not part of this rollout (the planar state has no
    lateral velocity); its weight must be zero.
  * Goal terms (Eq. 12): g = |mu_XY(k+1) - goal| at every stage, weight
    beta_2; F = P_goal * 1[|mu_XY(T) - goal| > goal_radius] on the last stage
    only, weight beta_3.
  * Terrain ensemble (Eq. 3): mean sum_i w_i m_i, variance sum_i w_i^2 var_i
    per output; M = 1, w = 1 is the single GP.
  * MPPI weights (Alg. 1, deferred to the MPPI reference): w = softmax of
    -(S - min S) / lambda; update U <- U + sum_s w_s (u~_s - U).
  * Variance mode 0 ("per sample") tightens each sample with its own
    propagated Sigma; mode 1 ("nominal", Alg. 1 Step 2) tightens every sample
    with the Sigma_XY(k+1) propagated along the previous update's U.
"""
from __future__ import annotations

import numpy as np

from .gp import predict
from .philox import control_noise
from .quantiles import chi2_2_quantile, normal_quantile

LANE_DISCOUNT = 0.9      # the 0.9^k factor of Eq. 11
RHO_EPS = 1e-9           # below this the obstacle normal of Eq. 15 is undefined


# --------------------------------------------------------------------------
# motion model: Eq. 1-2, Eq. 6, Eq. 10
# --------------------------------------------------------------------------

def nominal_step(mu, u, dt, tau_v, tau_w):
    """Nominal f(x, u) of Eq. 6 without the GP term; mu (...,5), u (...,2)."""
    X, Y, th, v, w = (mu[..., i] for i in range(5))
    return np.stack([
        X + dt * v * np.cos(th),
        Y + dt * v * np.sin(th),
        th + dt * w,
        v + (dt / tau_v) * (u[..., 0] - v),
        w + (dt / tau_w) * (u[..., 1] - w),
    ], axis=-1)


def jacobian(mu, dt, tau_v, tau_w):
    """d f / d mu of the nominal model at mu (...,5): (...,5,5)."""
    th, v = mu[..., 2], mu[..., 3]
    A = np.zeros(mu.shape[:-1] + (5, 5))
    for i in range(5):
        A[..., i, i] = 1.0
    A[..., 0, 2] = -dt * v * np.sin(th)
    A[..., 0, 3] = dt * np.cos(th)
    A[..., 1, 2] = dt * v * np.cos(th)
    A[..., 1, 3] = dt * np.sin(th)
    A[..., 2, 4] = dt
    A[..., 3, 3] = 1.0 - dt / tau_v
    A[..., 4, 4] = 1.0 - dt / tau_w
    return A


def covariance_step(Sig, A, var):
    """Eq. 10: Sigma' = A Sigma A^T + diag(0, 0, 0, var_v, var_omega)."""
    out = A @ Sig @ np.swapaxes(A, -1, -2)
    out[..., 3, 3] += var[..., 0]
    out[..., 4, 4] += var[..., 1]
    return out


# --------------------------------------------------------------------------
# costs and chance constraints: Eq. 11-16
# --------------------------------------------------------------------------

def lane_distance(p, path):
    """Euclidean distance from points p (S,2) to the polyline path (P,2)."""
    p = np.asarray(p, dtype=np.float64)
    path = np.asarray(path, dtype=np.float64)
    if path.shape[0] == 1:
        return np.hypot(p[:, 0] - path[0, 0], p[:, 1] - path[0, 1])
    a = path[:-1][None, :, :]                 # (1, P-1, 2)
    ab = (path[1:] - path[:-1])[None, :, :]
    ap = p[:, None, :] - a                    # (S, P-1, 2)
    len2 = np.sum(ab * ab, axis=-1)
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(len2 > 0.0, np.sum(ap * ab, axis=-1) / len2, 0.0)
    t = np.clip(t, 0.0, 1.0)
    q = ap - t[..., None] * ab
    return np.min(np.hypot(q[..., 0], q[..., 1]), axis=1)


def lambda_max_2x2(Sxy):
    """Largest eigenvalue of symmetric 2x2 blocks (...,2,2)."""
    return np.linalg.eigvalsh(Sxy)[..., -1]


def tightening_constants(p_x):
    """(sqrt(chi^2_2(p_x)), Phi^-1(p_x)) for Eq. 14 and Eq. 16."""
    return np.sqrt(chi2_2_quantile(p_x)), normal_quantile(p_x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * np.asarray(x, dtype=np.float64)))


def stage_cost(k, mu, Sxy, var, sc, consts, slope=None):
    """Stage cost c_track + c_avoidance at stage k.

    slope=None uses the indicators of Eq. 11-12; a positive slope replaces
    them by logistic sigmoids of slope * margin (lane) and -slope * margin
    (collision), the smooth surrogate the gradient is taken of.

    mu (S,5) is the state after the update of step k, Sxy (S,2,2) the
    position covariance used for tightening, var (S,2) the GP variance of
    that update.  Returns (cost, lane_margin, obstacle_margin), each (S,);
    the lane indicator fires when lane_margin > 0, the collision indicator
    when obstacle_margin <= 0 (+inf when there are no obstacles).
    """
    P = sc.params
    sq_chi2, phi_inv = consts
    trC = var[:, 0] + var[:, 1]
    lmax = np.maximum(lambda_max_2x2(Sxy), 0.0)
    r = P.lane_half_width
    r_bar = r - sq_chi2 * np.sqrt(lmax)                       # Eq. 14
    e = lane_distance(mu[:, :2], sc.path)
    lane_margin = e - r_bar
    lane_viol = (lane_margin > 0.0).astype(np.float64) if slope is None else sigmoid(slope * lane_margin)
    a = P.alpha
    cost = (a[0] * trC + a[1] * e / r
            + a[3] * P.P_lane * LANE_DISCOUNT ** k * lane_viol      # Eq. 11
            + a[4] * (P.v_desired - mu[:, 3]) ** 2)
    O = sc.obstacles.shape[0]
    if O > 0:
        delta = mu[:, None, :2] - sc.obstacles[None, :, :2]          # (S,O,2)
        rho = np.hypot(delta[..., 0], delta[..., 1])
        d = rho - sc.obstacles[None, :, 2]                            # signed distance
        safe = np.where(rho > RHO_EPS, rho, 1.0)
        n = delta / safe[..., None]                                   # Eq. 15
        nSn = np.einsum("soi,sij,soj->so", n, Sxy, n)
        spread = np.where(rho > RHO_EPS, np.sqrt(np.maximum(nSn, 0.0)),
                          np.sqrt(lmax)[:, None])
        d_bar = d - phi_inv * spread                                  # Eq. 16
        obs_margin = np.min(d_bar, axis=1)
    else:
        obs_margin = np.full(mu.shape[0], np.inf)
    if slope is None:
        coll = (obs_margin <= 0.0).astype(np.float64)
    else:
        coll = sigmoid(-slope * obs_margin) if O > 0 else np.zeros_like(obs_margin)
    b = P.beta
    cost = cost + b[0] * trC + b[1] * P.P_coll * coll                 # Eq. 12
    if b[2] != 0.0 or b[3] != 0.0:
        dg = np.hypot(mu[:, 0] - P.goal[0], mu[:, 1] - P.goal[1])
        cost = cost + b[2] * dg                                       # g, every stage
        if k == P.T - 1:                                              # F, terminal stage
            miss = (dg > P.goal_radius).astype(np.float64) if slope is None \
                else sigmoid(slope * (dg - P.goal_radius))
            cost = cost + b[3] * P.P_goal * miss
    return cost, lane_margin, obs_margin


# --------------------------------------------------------------------------
# Alg. 1 Step 1: sampled rollouts
# --------------------------------------------------------------------------

def _check_params(P):
    if P.alpha[2] != 0.0:
        raise ValueError("the slip term (alpha_2) is not modelled")


def rollout(sc, fits, state, U, it, samples=None, nominal_sxy=None, noise=True, slope=None):
    """Alg. 1 Step 1 for the listed samples (all K by default).

    state (5,), U (T,2), it the MPPI iteration (Philox counter words 2-3).
    nominal_sxy (T,2,2) replaces the per-sample Sigma_XY in the tightening
    (variance mode 1); None means per-sample tightening.
    Returns a dict with costs (S,), u_tilde (S,T,2), mu (S,T,5) (states after
    each step), Sigma (S,T,5,5), var (S,T,2), mean (S,T,2), stage (S,T),
    lane_margin and obs_margin (S,T).
    """
    P = sc.params
    _check_params(P)
    K, T = P.K, P.T
    s_idx = np.arange(K) if samples is None else np.asarray(samples, dtype=np.int64)
    S = s_idx.shape[0]
    consts = tightening_constants(P.p_x)
    umin, umax = np.asarray(P.u_min), np.asarray(P.u_max)
    mu = np.tile(np.asarray(state, dtype=np.float64), (S, 1))
    Sig = np.zeros((S, 5, 5))
    out = dict(costs=np.zeros(S), u_tilde=np.zeros((S, T, 2)), mu=np.zeros((S, T, 5)),
               Sigma=np.zeros((S, T, 5, 5)), var=np.zeros((S, T, 2)),
               mean=np.zeros((S, T, 2)), stage=np.zeros((S, T)),
               lane_margin=np.zeros((S, T)), obs_margin=np.zeros((S, T)))
    for k in range(T):
        eps = control_noise(P.seed, k, s_idx, it, P.sigma) if noise else np.zeros((S, 2))
        ut = np.clip(np.asarray(U[k], dtype=np.float64) + eps, umin, umax)   # Eq. 8
        z = np.stack([mu[:, 3], mu[:, 4], ut[:, 0], ut[:, 1]], axis=1)
        m, var = predict(fits, z)                                         # Eq. 3
        A = jacobian(mu, P.dt, P.tau_v, P.tau_w)
        mu = nominal_step(mu, ut, P.dt, P.tau_v, P.tau_w)                 # Eq. 6, 10
        mu[:, 3] += m[:, 0]
        mu[:, 4] += m[:, 1]
        Sig = covariance_step(Sig, A, var)                                # Eq. 10
        Sxy = Sig[:, :2, :2] if nominal_sxy is None else np.broadcast_to(nominal_sxy[k], (S, 2, 2))
        c, lm, om = stage_cost(k, mu, Sxy, var, sc, consts, slope)
        out["costs"] += c
        out["u_tilde"][:, k] = ut
        out["mu"][:, k] = mu
        out["Sigma"][:, k] = Sig
        out["var"][:, k] = var
        out["mean"][:, k] = m
        out["stage"][:, k] = c
        out["lane_margin"][:, k] = lm
        out["obs_margin"][:, k] = om
    return out


def mppi_weights(costs, lam):
    """Softmax of -(S - min S)/lambda (log-sum-exp shift by the minimum)."""
    costs = np.asarray(costs, dtype=np.float64)
    e = np.exp(-(costs - np.min(costs)) / lam)
    return e / np.sum(e)


def mppi_update(U, u_tilde, w):
    """U <- U + sum_s w_s (u~_s - U)  (Alg. 1 'weighted sum')."""
    U = np.asarray(U, dtype=np.float64)
    return U + np.einsum("s,skc->kc", w, u_tilde - U[None])


def nominal_tightening(sc, fits, state, U):
    """Alg. 1 Step 2: propagate mean and Sigma (Eq. 10) along U without noise
    and return Sigma_XY(k+1) for k = 0..T-1, shape (T,2,2)."""
    P = sc.params
    mu = np.asarray(state, dtype=np.float64)[None]
    Sig = np.zeros((1, 5, 5))
    umin, umax = np.asarray(P.u_min), np.asarray(P.u_max)
    out = np.zeros((P.T, 2, 2))
    for k in range(P.T):
        u = np.clip(np.asarray(U[k], dtype=np.float64), umin, umax)[None]
        z = np.stack([mu[:, 3], mu[:, 4], u[:, 0], u[:, 1]], axis=1)
        m, var = predict(fits, z)
        A = jacobian(mu, P.dt, P.tau_v, P.tau_w)
        mu = nominal_step(mu, u, P.dt, P.tau_v, P.tau_w)
        mu[:, 3] += m[:, 0]
        mu[:, 4] += m[:, 1]
        Sig = covariance_step(Sig, A, var)
        out[k] = Sig[0, :2, :2]
    return out


def mppi_step(sc, fits, state, U, it, nominal_sxy=None):
    """One MPPI iteration: rollout, weights, update.  Returns (U_new, w, costs, rollout)."""
    ro = rollout(sc, fits, state, U, it, nominal_sxy=nominal_sxy)
    w = mppi_weights(ro["costs"], sc.params.lam)
    return mppi_update(U, ro["u_tilde"], w), w, ro["costs"], ro


class Controller:
    """Receding-horizon use of Alg. 1: an iteration counter that advances per
    call and, in variance mode 1, the Step 2 tightening carried to the next call."""

    def __init__(self, sc, fits, it=0):
        self.sc, self.fits, self.it = sc, fits, int(it)
        self.nominal_sxy = np.zeros((sc.params.T, 2, 2)) if sc.params.variance_mode == 1 else None

    def step(self, state, U):
        U_new, w, costs, ro = mppi_step(self.sc, self.fits, state, U, self.it, self.nominal_sxy)
        if self.nominal_sxy is not None:
            self.nominal_sxy = nominal_tightening(self.sc, self.fits, state, U_new)
        self.it += 1
        return U_new, w, costs, ro


def plant_step(sc, state, u, residual):
    """Simulated robot: nominal model plus the true residual (closed-loop harness)."""
    P = sc.params
    u = np.clip(np.asarray(u, dtype=np.float64), P.u_min, P.u_max)
    nxt = nominal_step(np.asarray(state, dtype=np.float64), u, P.dt, P.tau_v, P.tau_w)
    d = residual(state[3], state[4], u[0], u[1])
    nxt[3] += d[0]
    nxt[4] += d[1]
    return nxt


def shift_controls(U):
    """Receding-horizon shift: drop the applied control, repeat the last one."""
    return np.concatenate([U[1:], U[-1:]], axis=0)
