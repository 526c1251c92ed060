"""Terrain-weight estimation, Eq. 4 (Alg. 1 Step 3), oracle side.

TEST INFRASTRUCTURE ONLY (see the package docstring).

    w* = argmin_w |Y_v - F_v w|^2 + |Y_w - F_w w|^2 + gamma |w - w_prev|_1
         s.t. 0 <= w_i <= 1, sum_i w_i = 1

Y_v, Y_w (H,) are the velocity residuals observed over the last H steps and
F_v, F_w (H, M) the M terrain GPs' mean predictions at the same inputs.  The
oracle solves the smooth equivalent with t_i >= |w_i - w_prev_i| as extra
variables by sequential least squares (scipy SLSQP) from several starting
points and keeps the best; it is a plain restatement of the problem, not the
method the library uses.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize


def terrain_objective(w, Yv, Yw, Fv, Fw, w_prev, gamma):
    w = np.asarray(w, dtype=np.float64)
    rv = Yv - Fv @ w
    rw = Yw - Fw @ w
    return float(rv @ rv + rw @ rw + gamma * np.sum(np.abs(w - w_prev)))


def terrain_weights(Yv, Yw, Fv, Fw, w_prev, gamma):
    Yv, Yw = np.asarray(Yv, float), np.asarray(Yw, float)
    Fv, Fw = np.asarray(Fv, float), np.asarray(Fw, float)
    w_prev = np.asarray(w_prev, float)
    M = Fv.shape[1]
    Q = Fv.T @ Fv + Fw.T @ Fw
    c = Fv.T @ Yv + Fw.T @ Yw

    def f(x):
        w, t = x[:M], x[M:]
        return float(w @ Q @ w - 2 * c @ w + gamma * np.sum(t))

    def g(x):
        w = x[:M]
        return np.concatenate([2 * Q @ w - 2 * c, np.full(M, gamma)])

    cons = [{"type": "eq", "fun": lambda x: np.sum(x[:M]) - 1.0, "jac": lambda x: np.r_[np.ones(M), np.zeros(M)]},
            {"type": "ineq", "fun": lambda x: x[M:] - (x[:M] - w_prev),
             "jac": lambda x: np.c_[-np.eye(M), np.eye(M)]},
            {"type": "ineq", "fun": lambda x: x[M:] + (x[:M] - w_prev),
             "jac": lambda x: np.c_[np.eye(M), np.eye(M)]}]
    bounds = [(0.0, 1.0)] * M + [(0.0, None)] * M
    starts = [w_prev, np.full(M, 1.0 / M)] + [np.eye(M)[i] for i in range(M)]
    best = None
    for w0 in starts:
        x0 = np.r_[w0, np.abs(w0 - w_prev)]
        r = minimize(f, x0, jac=g, bounds=bounds, constraints=cons, method="SLSQP",
                     options={"ftol": 1e-15, "maxiter": 1000})
        w = np.clip(r.x[:M], 0.0, 1.0)
        w = w / np.sum(w)
        val = terrain_objective(w, Yv, Yw, Fv, Fw, w_prev, gamma)
        if best is None or val < best[1]:
            best = (w, val)
    return best[0]
