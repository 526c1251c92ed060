"""Helpers for comparing the CUDA path with the FP64 oracle (test infrastructure).

Tolerances (the first three are the stated targets of this rollout):
  * trajectories (means) and costs: |gpu - ref| <= 1e-4 (|ref| + 1), i.e.
    1e-4 relative with a unit floor (metres, radians, m/s, cost units);
  * updated controls U_new: 1e-4 absolute;
  * weights: 1e-4 absolute (they lie in [0, 1] and sum to 1);
  * GP variance and covariance entries: |gpu - ref| <= 1e-4 sf2 per variance
    and 1e-4 (|ref| + sf2 (1 + T dt)) for Sigma, from the FP32 error bound of
    |L^-1 k*|^2 (about sqrt(N) eps32 |L^-1| |k*| |v|, i.e. a few 1e-5 sf2);
    Eq. 10 adds each step's GP variance to Sigma_vv and Sigma_ww, so the
    covariance floor is at least the variance's own scale sf2.

Indicators (Eq. 11, 12) are discontinuous: an FP32 trajectory and the FP64
one may fall on opposite sides of a boundary.  A stage whose FP64 margin lies
within MARGIN_WINDOW of zero is "ambiguous"; for a sample with ambiguous
stages the GPU cost must equal the oracle cost plus the penalties of some
subset of flipped indicators, and the oracle's update is then recomputed with
that valid alternative.  All other indicator decisions must agree exactly.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle as O

TOL_TRAJ = 1e-4
TOL_COST = 1e-4
TOL_U = 1e-4
TOL_W = 1e-4
# Margins e - r + sqrt(chi2) sqrt(lambda_max(Sigma_XY)) pass covariance errors
# through a square root: d sqrt(lambda) = d lambda / (2 sqrt(lambda)), a factor
# of up to ~10 at the covariance scales of these workloads, so margin values
# are held to 10x the trajectory tolerance; what they decide (indicator bits)
# is checked exactly outside MARGIN_WINDOW.
TOL_MARGIN = 1e-3
MARGIN_WINDOW = 2e-3      # metres
MAX_FLIPS = 12


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def make_ctrl(gp, sc, gpfit=None):
    """(GP handle(s), controller) for a scenario: its GP pair, or its terrain
    ensemble (Eq. 3) when the scenario has one."""
    if sc.terrains is not None:
        gps = [gp.gp_fit(X, Y, h) for X, Y, h in sc.terrains]
        return gps, gp.mppi_create_ensemble(sc.params, sc.obstacles, sc.path, gps, sc.terrain_w)
    g = gpfit if gpfit is not None else gp.gp_fit(sc.X, sc.Y, sc.hyper)
    return g, gp.mppi_create(sc.params, sc.obstacles, sc.path, g)


def signal_var(sc):
    """Largest prior variance of the scenario's GP(s): the scale of the variance tolerance."""
    if sc.terrains is not None:
        return max(h[0].signal_var for _, _, h in sc.terrains)
    return sc.hyper[0].signal_var


def gpu_step(gp, ctrl, sc, state, U, it=None):
    import torch
    dev = torch.device("cuda")
    if it is not None:
        gp.mppi_set_iteration(ctrl, it)
    Ud = torch.tensor(np.asarray(U), dtype=torch.float32, device=dev)
    U_new = torch.empty_like(Ud)
    w = torch.empty(sc.params.K, dtype=torch.float32, device=dev)
    c = torch.empty_like(w)
    gp.mppi_step(ctrl, state, Ud, U_new, w, c)
    gp.mppi_device_status(ctrl)        # no kernel gave up a bounded wait
    return to_np(U_new), to_np(w), to_np(c)


def gpu_trace(gp, ctrl, sc, state, U, it=None):
    import torch
    dev = torch.device("cuda")
    if it is not None:
        gp.mppi_set_iteration(ctrl, it)
    K, T = sc.params.K, sc.params.T
    Ud = torch.tensor(np.asarray(U), dtype=torch.float32, device=dev)
    mu = torch.empty(K, T, 5, device=dev)
    sig = torch.empty(K, T, 15, device=dev)
    st = torch.empty(K, T, device=dev)
    mg = torch.empty(K, T, 2, device=dev)
    c = torch.empty(K, device=dev)
    gp.mppi_rollout_trace(ctrl, state, Ud, mu, sig, st, mg, c)
    gp.mppi_device_status(ctrl)
    return dict(mu=to_np(mu), sigma=to_np(sig), stage=to_np(st), margins=to_np(mg), costs=to_np(c))


UPPER = [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3), (1, 4),
         (2, 2), (2, 3), (2, 4), (3, 3), (3, 4), (4, 4)]


def sigma_upper(S):
    """(..., 5, 5) -> (..., 15) in the ABI's upper-triangle order."""
    return np.stack([S[..., i, j] for i, j in UPPER], axis=-1)


def sig_floor(sc):
    """Covariance tolerance floor: the GP variance scale sf2 plus the growth of
    the position entries over the horizon."""
    return signal_var(sc) * (1.0 + sc.params.T * sc.params.dt)


def close(gpu, ref, rtol, floor=1.0):
    return np.abs(gpu - ref) <= rtol * (np.abs(ref) + floor)


def assert_close(gpu, ref, rtol, floor=1.0, what=""):
    ok = close(gpu, ref, rtol, floor)
    if not np.all(ok):
        idx = np.argwhere(~ok)[:5]
        err = np.max(np.abs(gpu - ref) / (np.abs(ref) + floor))
        raise AssertionError(f"{what}: {np.sum(~ok)} / {ok.size} outside tolerance {rtol} "
                             f"(max scaled err {err:.3e}); first {idx.tolist()}")


def _penalties(sc):
    P = sc.params
    return P.alpha[3] * P.P_lane, P.beta[1] * P.P_coll


def reconcile_costs(sc, ro, gpu_costs, rows=None):
    """Indicator-tie protocol.  Returns (adjusted oracle costs, number of
    samples whose cost was taken from a valid alternative)."""
    c_lane, c_coll = _penalties(sc)
    P = sc.params
    ref = ro["costs"].copy()
    lm, om = ro["lane_margin"], ro["obs_margin"]
    T = lm.shape[1]
    disc = 0.9 ** np.arange(T)
    c_term = P.beta[3] * P.P_goal
    # terminal goal indicator (Eq. 12 F): distance of the final mean beyond the radius
    gm = np.hypot(ro["mu"][:, T - 1, 0] - P.goal[0], ro["mu"][:, T - 1, 1] - P.goal[1]) - P.goal_radius
    n_alt = 0
    for s in range(ref.shape[0]):
        if close(gpu_costs[s], ref[s], TOL_COST):
            continue
        deltas = []
        if c_term != 0.0 and abs(gm[s]) < MARGIN_WINDOW:
            deltas.append(-c_term if gm[s] > 0 else c_term)
        for k in range(T):
            if abs(lm[s, k]) < MARGIN_WINDOW and c_lane != 0.0:
                sign = -1.0 if lm[s, k] > 0 else 1.0
                deltas.append(sign * c_lane * disc[k])
            if np.isfinite(om[s, k]) and abs(om[s, k]) < MARGIN_WINDOW and c_coll != 0.0:
                sign = -1.0 if om[s, k] <= 0 else 1.0
                deltas.append(sign * c_coll)
        found = False
        if deltas and len(deltas) <= MAX_FLIPS:
            for r in range(1, len(deltas) + 1):
                for comb in itertools.combinations(deltas, r):
                    alt = ref[s] + sum(comb)
                    if close(gpu_costs[s], alt, TOL_COST):
                        ref[s] = alt
                        found = True
                        break
                if found:
                    break
        if not found:
            who = s if rows is None else rows[s]
            raise AssertionError(f"sample {who}: gpu cost {gpu_costs[s]:.6f} vs oracle {ro['costs'][s]:.6f} "
                                 f"and no valid indicator flip explains it ({len(deltas)} ambiguous stages)")
        n_alt += 1
    return ref, n_alt


def check_step(sc, ro, U, gpu_U_new, gpu_w, gpu_c):
    """Full-step parity: costs (with the tie protocol), weights, U_new."""
    ref_c, n_alt = reconcile_costs(sc, ro, gpu_c)
    assert_close(gpu_c, ref_c, TOL_COST, what="costs")
    w = O.mppi_weights(ref_c, sc.params.lam)
    U_ref = O.mppi_update(U, ro["u_tilde"], w)
    err_w = np.max(np.abs(gpu_w - w))
    err_u = np.max(np.abs(gpu_U_new - U_ref))
    assert err_w <= TOL_W, f"weights max abs err {err_w:.3e}"
    assert err_u <= TOL_U, f"U_new max abs err {err_u:.3e}"
    return dict(n_alt=n_alt, err_w=err_w, err_u=err_u,
                err_c=float(np.max(np.abs(gpu_c - ref_c) / (np.abs(ref_c) + 1.0))))


def check_trace(sc, ro, tr, rows=None):
    """Per-(sample, step) parity of means, covariances, stage costs, margins."""
    rows = np.arange(ro["costs"].shape[0]) if rows is None else np.asarray(rows)
    mu_g = tr["mu"][rows]
    assert_close(mu_g, ro["mu"], TOL_TRAJ, what="trajectory means")
    sig_ref = sigma_upper(ro["Sigma"])
    assert_close(tr["sigma"][rows], sig_ref, TOL_TRAJ, floor=sig_floor(sc), what="covariances")
    # margins: continuous quantities
    mg = tr["margins"][rows]
    assert_close(mg[..., 0], ro["lane_margin"], TOL_MARGIN, what="lane margins")
    om = ro["obs_margin"]
    if np.all(np.isinf(om)):
        assert np.all(np.isinf(mg[..., 1]))
    else:
        assert_close(mg[..., 1], om, TOL_MARGIN, what="obstacle margins")
    # indicator bits agree wherever the oracle's margin is clear of the boundary
    clear_l = np.abs(ro["lane_margin"]) >= MARGIN_WINDOW
    assert np.array_equal((mg[..., 0] > 0)[clear_l], (ro["lane_margin"] > 0)[clear_l])
    clear_o = np.isfinite(om) & (np.abs(om) >= MARGIN_WINDOW)
    assert np.array_equal((mg[..., 1] <= 0)[clear_o], (om <= 0)[clear_o])
    n_amb = int(np.sum(~clear_l) + np.sum(np.isfinite(om) & ~clear_o))
    lm_err = float(np.max(np.abs(mg[..., 0] - ro["lane_margin"]) / (np.abs(ro["lane_margin"]) + 1)))
    return dict(n_ambiguous_stages=n_amb, err_lane_margin=lm_err,
                err_mu=float(np.max(np.abs(mu_g - ro["mu"]) / (np.abs(ro["mu"]) + 1))),
                err_sigma=float(np.max(np.abs(tr["sigma"][rows] - sig_ref)
                                       / (np.abs(sig_ref) + sig_floor(sc)))))


def trace_errors(sc, ro, tr, rows=None):
    """Max scaled errors per quantity (no assertion): means, covariances,
    lane margins (with the floors of the parity tolerances)."""
    rows = np.arange(ro["costs"].shape[0]) if rows is None else np.asarray(rows)
    sig_ref = sigma_upper(ro["Sigma"])
    mg = tr["margins"][rows]
    return dict(
        err_mu=float(np.max(np.abs(tr["mu"][rows] - ro["mu"]) / (np.abs(ro["mu"]) + 1))),
        err_sigma=float(np.max(np.abs(tr["sigma"][rows] - sig_ref) / (np.abs(sig_ref) + sig_floor(sc)))),
        err_lane_margin=float(np.max(np.abs(mg[..., 0] - ro["lane_margin"]) / (np.abs(ro["lane_margin"]) + 1))))
