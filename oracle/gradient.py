"""Gradient of the smoothed chance-constrained MPPI objective (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The objective is the sample mean of the rollout costs with the lane and
collision indicators of Eq. 11-12 replaced by logistic sigmoids of slope *
margin, J(U, l) = (1/S) sum_s S_s(U, l), with the control noise held fixed
(same Philox draws).  Its gradient with respect to the nominal controls U
and the SE-ARD lengthscales l of the two residual GPs (which enter the
kernel rows and, through the fit, alpha = K^-1 y and L^-1) is the plain
definition: central differences in FP64.
"""
from __future__ import annotations

import copy

import numpy as np

from .gp import gp_fit
from .mppi import rollout


def objective(sc, hypers, state, U, it, samples, slope, fits=None):
    """J = mean over the listed samples of the smoothed rollout costs."""
    if fits is None:
        fits = gp_fit(sc.X, sc.Y, hypers)
    ro = rollout(sc, fits, state, U, it, samples=samples, slope=slope)
    return float(np.mean(ro["costs"])), ro


def with_lengthscale(hypers, o, d, delta):
    """Copy of the hyper-parameter pair with l_{o,d} moved by delta."""
    out = [copy.deepcopy(hypers[0]), copy.deepcopy(hypers[1])]
    ell = list(out[o].lengthscale)
    ell[d] += delta
    out[o].lengthscale = tuple(ell)
    return tuple(out)


def fd_gradient(sc, hypers, state, U, it, samples, slope, h_u=1e-6, h_l=1e-6, ell=True):
    """Central differences of J: (dJ/dU (T,2), dJ/dl (2,4) or None)."""
    U = np.asarray(U, dtype=np.float64)
    fits = gp_fit(sc.X, sc.Y, hypers)
    gU = np.zeros_like(U)
    for k in range(U.shape[0]):
        for c in range(2):
            Up, Um = U.copy(), U.copy()
            Up[k, c] += h_u
            Um[k, c] -= h_u
            jp, _ = objective(sc, hypers, state, Up, it, samples, slope, fits)
            jm, _ = objective(sc, hypers, state, Um, it, samples, slope, fits)
            gU[k, c] = (jp - jm) / (2 * h_u)
    gL = None
    if ell:
        gL = np.zeros((2, 4))
        for o in range(2):
            for d in range(4):
                jp, _ = objective(sc, with_lengthscale(hypers, o, d, h_l), state, U, it, samples, slope)
                jm, _ = objective(sc, with_lengthscale(hypers, o, d, -h_l), state, U, it, samples, slope)
                gL[o, d] = (jp - jm) / (2 * h_l)
    return gU, gL
