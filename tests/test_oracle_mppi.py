"""Pins for the oracle's MPPI weights / update (Alg. 1) and the nominal mode."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from test_oracle_dynamics import lab


def test_weights_sum_to_one_and_shift_invariant():
    rng = np.random.default_rng(0)
    c = rng.uniform(0, 50, 1000)
    w = O.mppi_weights(c, 1.0)
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(O.mppi_weights(c + 1234.5, 1.0), w, rtol=1e-10)
    # plain softmax where it does not overflow
    e = np.exp(-c / 3.0)
    np.testing.assert_allclose(O.mppi_weights(c, 3.0), e / e.sum(), rtol=1e-12)


def test_temperature_limits():
    c = np.array([3.0, 1.0, 2.0, 1.5])
    w0 = O.mppi_weights(c, 1e-6)
    np.testing.assert_allclose(w0, [0, 1, 0, 0], atol=1e-100)
    winf = O.mppi_weights(c, 1e12)
    np.testing.assert_allclose(winf, 0.25, rtol=1e-10)
    # exact ties share the weight equally
    np.testing.assert_allclose(O.mppi_weights(np.array([1.0, 1.0, 5.0]), 1e-6), [0.5, 0.5, 0.0], atol=1e-100)


def test_update_single_sample_and_permutation():
    rng = np.random.default_rng(1)
    U = rng.standard_normal((6, 2))
    ut = rng.standard_normal((1, 6, 2))
    np.testing.assert_allclose(O.mppi_update(U, ut, np.array([1.0])), ut[0], rtol=0, atol=1e-15)
    ut = rng.standard_normal((9, 6, 2))
    w = O.mppi_weights(rng.uniform(0, 3, 9), 1.0)
    perm = rng.permutation(9)
    np.testing.assert_allclose(O.mppi_update(U, ut[perm], w[perm]), O.mppi_update(U, ut, w), rtol=1e-13)


def test_full_step_properties():
    sc = S.scenario("small")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U_new, w, costs, ro = O.mppi_step(sc, fits, sc.x0, sc.U0, it=0)
    P = sc.params
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.all(U_new >= np.array(P.u_min) - 1e-15) and np.all(U_new <= np.array(P.u_max) + 1e-15)
    # subset of samples = same rows of the full rollout (samples are independent)
    sub = O.rollout(sc, fits, sc.x0, sc.U0, it=0, samples=[3, 70, 11])
    # (BLAS blocking may differ with the batch size: agree to rounding)
    np.testing.assert_allclose(sub["costs"], ro["costs"][[3, 70, 11]], rtol=1e-13)
    np.testing.assert_allclose(sub["mu"], ro["mu"][[3, 70, 11]], rtol=1e-13, atol=1e-15)
    # the iteration counter changes the draws
    ro2 = O.rollout(sc, fits, sc.x0, sc.U0, it=1)
    assert not np.allclose(ro2["u_tilde"], ro["u_tilde"])


def test_clamped_controls_inside_box():
    sc = S.scenario("small")
    sc.params.sigma = (5.0, 5.0)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, it=0)
    ut = ro["u_tilde"]
    assert np.any(ut[..., 0] == 0.0) and np.any(ut[..., 0] == 2.0)
    assert ut.min() >= -1.5 and ut.max() <= 2.0


def test_nominal_mode_equals_per_sample_without_noise():
    # with zero sampling noise every sample follows the nominal trajectory, so
    # tightening with the Step 2 covariance along U equals per-sample tightening
    sc = S.scenario("small")
    sc.params.sigma = (0.0, 0.0)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = sc.U0.copy()
    U[:, 1] = 0.3
    sxy = O.nominal_tightening(sc, fits, sc.x0, U)
    a = O.rollout(sc, fits, sc.x0, U, it=0)
    b = O.rollout(sc, fits, sc.x0, U, it=0, nominal_sxy=sxy)
    np.testing.assert_allclose(b["costs"], a["costs"], rtol=1e-13)
    np.testing.assert_allclose(sxy, a["Sigma"][0, :, :2, :2], rtol=1e-13, atol=1e-18)


def test_controller_closed_loop_tracks_straight_path():
    sc = S.scenario("cfg1", K=128)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ctl = O.Controller(sc, fits)
    x, U = sc.x0.copy(), sc.U0.copy()
    ys = []
    for _ in range(40):
        U_new, w, costs, _ = ctl.step(x, U)
        x = O.mppi.plant_step(sc, x, U_new[0], S.true_residual)
        U = O.mppi.shift_controls(U_new)
        ys.append(x[1])
    assert ctl.it == 40
    assert x[0] > 1.5                     # moved forward along the path
    assert np.max(np.abs(ys)) < sc.params.lane_half_width
