"""Pins for the oracle's costs and chance-constraint tightening (Eq. 11-16)."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from test_oracle_dynamics import lab

SQ_CHI2 = 2.447746830680816       # sqrt(chi^2_2(0.95)), standard tables
PHI_INV = 1.6448536269514722      # Phi^-1(0.95), standard tables


def test_lane_distance_against_dense_sampling():
    rng = np.random.default_rng(0)
    path = S.path_figure_eight(5.0, 64)
    pts = rng.uniform(-7, 7, size=(200, 2))
    # dense points on every segment; the exact distance is at most the sampled one
    t = np.linspace(0, 1, 4001)[None, :, None]
    dense = (path[:-1, None, :] + t * (path[1:, None, :] - path[:-1, None, :])).reshape(-1, 2)
    brute = np.min(np.hypot(pts[:, None, 0] - dense[None, :, 0], pts[:, None, 1] - dense[None, :, 1]), axis=1)
    e = O.lane_distance(pts, path)
    assert np.all(e <= brute + 1e-12)
    seg = np.max(np.hypot(*(path[1:] - path[:-1]).T))
    assert np.all(brute - e <= seg / 4000 + 1e-12)


def test_lane_distance_straight_and_endpoints():
    path = np.array([[0.0, 0.0], [10.0, 0.0]])
    p = np.array([[3.0, 2.0], [-3.0, 4.0], [13.0, -4.0], [5.0, 0.0]])
    np.testing.assert_allclose(O.lane_distance(p, path), [2.0, 5.0, 5.0, 0.0], rtol=1e-15)
    # degenerate segment and single-point path
    np.testing.assert_allclose(O.lane_distance(p[:1], np.array([[1.0, 1.0], [1.0, 1.0]])), [np.hypot(2, 1)])
    np.testing.assert_allclose(O.lane_distance(p[:1], np.array([[1.0, 1.0]])), [np.hypot(2, 1)])


def test_lambda_max_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, c = rng.uniform(0, 2, 2)
        b = rng.uniform(-1, 1)
        ref = 0.5 * (a + c) + np.hypot(0.5 * (a - c), b)
        assert O.lambda_max_2x2(np.array([[a, b], [b, c]])) == pytest.approx(ref, rel=1e-13)


def test_isotropic_tightening():
    # Sigma_XY = s^2 I  =>  r_bar = r - 2.4477 s  and  d_bar = d - 1.6449 s
    sc = S.scenario("small", O=1, path="straight")
    sc = sc.replace(obstacles=np.array([[5.0, 3.0, 0.5]]))
    s = 0.2
    mu = np.array([[5.0, 0.7, 0.0, 1.5, 0.0]])
    Sxy = np.array([s * s * np.eye(2)])
    c, lm, om = O.stage_cost(0, mu, Sxy, np.zeros((1, 2)), sc, O.mppi.tightening_constants(0.95))
    r = sc.params.lane_half_width
    assert lm[0] == pytest.approx(0.7 - (r - SQ_CHI2 * s), rel=1e-13)
    assert om[0] == pytest.approx((3.0 - 0.7 - 0.5) - PHI_INV * s, rel=1e-13)


def test_directional_obstacle_spread():
    # anisotropic Sigma: only the variance along the normal n enters Eq. 16
    sc = S.scenario("small", O=1, path="straight")
    sc = sc.replace(obstacles=np.array([[0.0, 4.0, 1.0]]))
    mu = np.array([[0.0, 0.0, 0.0, 1.5, 0.0]])
    Sxy = np.array([[[0.25, 0.0], [0.0, 0.04]]])     # n = (0, -1): spread 0.2
    _, _, om = O.stage_cost(3, mu, Sxy, np.zeros((1, 2)), sc, O.mppi.tightening_constants(0.95))
    assert om[0] == pytest.approx(3.0 - PHI_INV * 0.2, rel=1e-13)


def _geom_v(P, v0, vc):
    a = 1.0 - P.dt / P.tau_v
    return vc + (v0 - vc) * a ** np.arange(1, P.T + 1)   # v(1) .. v(T)


def test_straight_path_speed_cost_closed_form():
    sc = lab(T=20, path="straight")
    P = sc.params
    x0 = np.array([0.0, 0.0, 0.0, 0.5, 0.0])
    U = np.tile([1.0, 0.0], (P.T, 1))
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, x0, U, it=0)
    v = _geom_v(P, 0.5, 1.0)
    ref = np.sum(P.alpha[4] * (P.v_desired - v) ** 2)
    assert ro["costs"][0] == pytest.approx(ref, rel=1e-13)


def test_lane_indicator_discount_closed_form():
    # path offset by 2 m from the robot's line: e = 2 > r_bar = r every stage
    sc = lab(T=20, path="straight")
    sc = sc.replace(path=np.array([[-10.0, 2.0], [50.0, 2.0]]))
    P = sc.params
    x0 = np.array([0.0, 0.0, 0.0, 0.5, 0.0])
    U = np.tile([1.0, 0.0], (P.T, 1))
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, x0, U, it=0)
    v = _geom_v(P, 0.5, 1.0)
    k = np.arange(P.T)
    ref = np.sum(P.alpha[1] * 2.0 / P.lane_half_width + P.alpha[3] * P.P_lane * 0.9 ** k
                 + P.alpha[4] * (P.v_desired - v) ** 2)
    assert ro["costs"][0] == pytest.approx(ref, rel=1e-13)


def test_collision_indicator_closed_form():
    # obstacle on the robot's straight line: stages whose position lies within
    # the radius count beta_1 * P_coll (Sigma = 0, so d_bar = d)
    sc = lab(T=30, path="straight")
    xc, R = 0.613, 0.25
    sc = sc.replace(obstacles=np.array([[xc, 0.0, R]]))
    P = sc.params
    x0 = np.array([0.0, 0.0, 0.0, 1.0, 0.0])
    U = np.tile([1.0, 0.0], (P.T, 1))
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, x0, U, it=0)
    X = P.dt * np.arange(1, P.T + 1) * 1.0           # v stays at 1
    hits = np.abs(X - xc) - R <= 0.0
    assert hits.sum() > 0
    ref = np.sum(P.beta[1] * P.P_coll * hits + P.alpha[4] * (P.v_desired - 1.0) ** 2)
    assert ro["costs"][0] == pytest.approx(ref, rel=1e-13)
    np.testing.assert_allclose(ro["obs_margin"][0], np.abs(X - xc) - R, atol=1e-13)


def test_variance_cost_term():
    # far training set: GP variance = sf2 for both outputs at every stage
    sf2 = 0.04
    sc = lab(T=10, sf2=sf2, far=True, path="straight")
    sc = sc.replace(path=np.array([[-10.0, 0.0], [50.0, 0.0]]))
    sc.params.alpha = (1.0, 0.0, 0.0, 0.0, 0.0)
    sc.params.beta = (0.5, 0.0, 0.0, 0.0)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, np.array([0, 0, 0, 1.0, 0]), np.tile([1.0, 0.0], (10, 1)), it=0)
    assert ro["costs"][0] == pytest.approx(10 * 1.5 * 2 * sf2, rel=1e-13)
