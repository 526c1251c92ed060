"""Gaussian-process residual model (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. III-A trains two GPs (one per velocity residual) on inputs
z = (v, omega, v_cmd, omega_cmd) and uses their predictive mean m and
covariance C inside Eq. 3 (one terrain, weight 1).  The kernel is the
squared-exponential with one lengthscale per input (ARD), zero prior mean:

    k(a, b) = sf2 * exp(-1/2 * sum_d (a_d - b_d)^2 / l_d^2)

and the standard GP regression posterior of the latent function (GP textbook,
Rasmussen & Williams Alg. 2.1):

    L = chol(K_XX + sn2 I),  alpha = K^-1 y = L^-T L^-1 y,
    m(z) = k(z, X) alpha,    var(z) = sf2 - || L^-1 k(X, z) ||^2,

clamped at zero from below (the exact value lies in [0, sf2]).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def se_ard(A, B, lengthscale, signal_var):
    """SE-ARD cross-covariance between rows of A (n,4) and B (m,4): (n, m)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ell = np.asarray(lengthscale, dtype=np.float64)
    d = (A[:, None, :] - B[None, :, :]) / ell
    return float(signal_var) * np.exp(-0.5 * np.sum(d * d, axis=-1))


def gp_fit(X, Y, hypers):
    """Fit the two residual GPs.  hypers: pair of objects with lengthscale,
    signal_var, noise_var.  Returns a list of per-output dicts."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    fits = []
    for j in range(2):
        h = hypers[j]
        Kxx = se_ard(X, X, h.lengthscale, h.signal_var)
        Kxx = Kxx + float(h.noise_var) * np.eye(X.shape[0])
        L = np.linalg.cholesky(Kxx)
        Linv = sla.solve_triangular(L, np.eye(X.shape[0]), lower=True)
        alpha = sla.cho_solve((L, True), Y[:, j])
        fits.append(dict(X=X, L=L, Linv=Linv, alpha=alpha,
                         lengthscale=np.asarray(h.lengthscale, dtype=np.float64),
                         signal_var=float(h.signal_var), noise_var=float(h.noise_var)))
    return fits


def gp_predict(fits, Z):
    """Latent predictive mean and variance at queries Z (M,4): each (M, 2)."""
    Z = np.asarray(Z, dtype=np.float64)
    mean = np.zeros((Z.shape[0], 2))
    var = np.zeros((Z.shape[0], 2))
    for j, f in enumerate(fits):
        if f["X"].shape[0] == 0:
            var[:, j] = f["signal_var"]
            continue
        Ks = se_ard(Z, f["X"], f["lengthscale"], f["signal_var"])     # (M, N)
        mean[:, j] = Ks @ f["alpha"]
        V = sla.solve_triangular(f["L"], Ks.T, lower=True)            # L^-1 k*, (N, M)
        var[:, j] = np.maximum(0.0, f["signal_var"] - np.sum(V * V, axis=0))
    return mean, var


class Ensemble:
    """Weighted terrain ensemble of Eq. 3: M fitted GP pairs and weights w."""

    def __init__(self, fits, w):
        self.fits = list(fits)
        self.w = np.asarray(w, dtype=np.float64)
        if len(self.fits) != self.w.shape[0]:
            raise ValueError("one weight per terrain")


def gp_predict_ensemble(ens, Z):
    """Eq. 3: mean sum_i w_i m_i(z), covariance sum_i w_i^2 C_i(z) (diagonal,
    the two outputs are independent GPs)."""
    Z = np.asarray(Z, dtype=np.float64)
    mean = np.zeros((Z.shape[0], 2))
    var = np.zeros((Z.shape[0], 2))
    for wi, f in zip(ens.w, ens.fits):
        m, v = gp_predict(f, Z)
        mean += wi * m
        var += wi * wi * v
    return mean, var


def predict(model, Z):
    """Mean and variance of the residual model: one GP pair or an Ensemble."""
    if isinstance(model, Ensemble):
        return gp_predict_ensemble(model, Z)
    return gp_predict(model, Z)


def fit_scenario(sc):
    """The residual model of a scenario: its GP pair, or its terrain ensemble."""
    if sc.terrains is None:
        return gp_fit(sc.X, sc.Y, sc.hyper)
    return Ensemble([gp_fit(X, Y, h) for X, Y, h in sc.terrains], sc.terrain_w)
