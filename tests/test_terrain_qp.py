"""The library's exact Eq. 4 solver (host code in the C-ABI library, no GPU
needed) against the oracle's SLSQP restatement."""
import numpy as np
import pytest

import oracle as O
from paper_2411_03289_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    import paper_2411_03289_gb300 as gp
    gp.load()
    return gp


def _problem(seed, H, M, noise):
    rng = np.random.default_rng(seed)
    Fv, Fw = rng.normal(size=(H, M)), rng.normal(size=(H, M))
    w_true = rng.dirichlet(np.ones(M))
    Yv = Fv @ w_true + noise * rng.normal(size=H)
    Yw = Fw @ w_true + noise * rng.normal(size=H)
    return Yv, Yw, Fv, Fw, rng.dirichlet(np.ones(M))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("M", [1, 2, 3, 5])
@pytest.mark.parametrize("gamma", [0.0, 0.3, 5.0])
def test_matches_oracle(lib, seed, M, gamma):
    Yv, Yw, Fv, Fw, w_prev = _problem(seed, 20, M, 0.3)
    w = lib.terrain_weights(Yv, Yw, Fv, Fw, w_prev, gamma)
    wo = O.terrain_weights(Yv, Yw, Fv, Fw, w_prev, gamma)
    assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-12
    f = O.terrain_objective(w, Yv, Yw, Fv, Fw, w_prev, gamma)
    fo = O.terrain_objective(wo, Yv, Yw, Fv, Fw, w_prev, gamma)
    # exact: never worse than the iterative oracle, and equal up to its tolerance
    assert f <= fo + 1e-9 * max(1.0, abs(fo))
    assert f >= fo - 1e-6 * max(1.0, abs(fo))
    np.testing.assert_allclose(w, wo, atol=2e-4)


def test_exact_recovery_and_limits(lib):
    Yv, Yw, Fv, Fw, w_prev = _problem(11, 30, 3, 0.0)
    w_true = O.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 0.0)
    np.testing.assert_allclose(lib.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 0.0), w_true, atol=1e-7)
    np.testing.assert_allclose(lib.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 1e7), w_prev, atol=1e-12)


def test_collinear_predictions(lib):
    """Two terrains predicting the same thing: a flat direction; any minimiser will do."""
    rng = np.random.default_rng(3)
    F = rng.normal(size=(15, 1))
    Fv = np.hstack([F, F, rng.normal(size=(15, 1))])
    Fw = np.hstack([F, F, rng.normal(size=(15, 1))])
    Yv, Yw = rng.normal(size=15), rng.normal(size=15)
    w_prev = np.array([0.2, 0.3, 0.5])
    w = lib.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 0.0)
    wo = O.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 0.0)
    f = O.terrain_objective(w, Yv, Yw, Fv, Fw, w_prev, 0.0)
    fo = O.terrain_objective(wo, Yv, Yw, Fv, Fw, w_prev, 0.0)
    assert f <= fo + 1e-9


def test_errors(lib):
    Yv, Yw, Fv, Fw, w_prev = _problem(1, 5, 3, 0.1)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.terrain_weights(Yv, Yw, Fv, Fw, w_prev, -1.0)
    assert ei.value.code == lib.GPMPPI_ERR_INVALID_ARG
    Fv2 = Fv.copy()
    Fv2[0, 0] = np.nan
    with pytest.raises(lib.GpmppiError) as ei:
        lib.terrain_weights(Yv, Yw, Fv2, Fw, w_prev, 0.1)
    assert ei.value.code == lib.GPMPPI_ERR_NONFINITE
    F9 = np.zeros((5, 9))
    with pytest.raises(lib.GpmppiError) as ei:
        lib.terrain_weights(Yv, Yw, F9, F9, np.full(9, 1 / 9), 0.1)
    assert ei.value.code == lib.GPMPPI_ERR_INVALID_ARG
