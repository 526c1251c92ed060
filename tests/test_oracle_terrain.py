"""Pins for the terrain ensemble (Eq. 3), the goal terms (Eq. 12) and the
terrain-weight estimation (Eq. 4) of the oracle."""
import itertools

import numpy as np
import pytest

import oracle as O
import scenarios as S


def _fits(seed, N=30, ell=0.5):
    rng = np.random.default_rng(seed)
    X, Y = S.gp_training_set(rng, N)
    h = S.Hyper((ell,) * 4, 0.1, 1e-4)
    return O.gp_fit(X, Y, (h, h))


def test_ensemble_single_and_one_hot():
    f = [_fits(1), _fits(2, ell=0.7), _fits(3, ell=0.4)]
    Z = np.random.default_rng(4).uniform([0, -1.5, 0, -1.5], [2, 1.5, 2, 1.5], (50, 4))
    m0, v0 = O.gp_predict(f[0], Z)
    m, v = O.predict(O.Ensemble([f[0]], [1.0]), Z)
    np.testing.assert_array_equal(m, m0)
    np.testing.assert_array_equal(v, v0)
    for i in range(3):
        mi, vi = O.gp_predict(f[i], Z)
        m, v = O.predict(O.Ensemble(f, np.eye(3)[i]), Z)
        np.testing.assert_allclose(m, mi, rtol=0, atol=1e-15)
        np.testing.assert_allclose(v, vi, rtol=0, atol=1e-15)


def test_ensemble_identical_terrains_square_weights():
    f = _fits(5)
    Z = np.random.default_rng(6).uniform([0, -1.5, 0, -1.5], [2, 1.5, 2, 1.5], (40, 4))
    m1, v1 = O.gp_predict(f, Z)
    w = np.array([0.5, 0.3, 0.2])
    m, v = O.predict(O.Ensemble([f, f, f], w), Z)
    np.testing.assert_allclose(m, m1, rtol=1e-13, atol=1e-16)
    # variances mix with the squared weights: 0.25 + 0.09 + 0.04 = 0.38
    np.testing.assert_allclose(v, 0.38 * v1, rtol=1e-13, atol=1e-18)


def test_ensemble_rollout_with_one_terrain_is_the_single_gp():
    sc = S.scenario("small")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    a = O.rollout(sc, fits, sc.x0, sc.U0, 0)
    b = O.rollout(sc, O.Ensemble([fits], [1.0]), sc.x0, sc.U0, 0)
    np.testing.assert_array_equal(a["costs"], b["costs"])
    np.testing.assert_array_equal(a["mu"], b["mu"])


def test_terrain_scenario_fit_matches_its_parts():
    sc = S.terrain_scenario("small", M=3, N=20)
    ens = O.fit_scenario(sc)
    assert isinstance(ens, O.Ensemble) and len(ens.fits) == 3
    assert ens.w.sum() == pytest.approx(1.0)
    Z = np.random.default_rng(1).uniform([0, -1.5, 0, -1.5], [2, 1.5, 2, 1.5], (10, 4))
    m, v = O.predict(ens, Z)
    parts = [O.gp_predict(O.gp_fit(X, Y, h), Z) for X, Y, h in sc.terrains]
    np.testing.assert_allclose(m, sum(w * p[0] for w, p in zip(ens.w, parts)), rtol=1e-12)
    np.testing.assert_allclose(v, sum(w * w * p[1] for w, p in zip(ens.w, parts)), rtol=1e-12)


def test_goal_terms_straight_line():
    """Zero noise, zero residual, heading 0, constant command u: v(k) relaxes to
    u geometrically and X(k+1) = X(k) + dt v(k), so the distance to a goal on
    the axis and the terminal indicator follow by hand."""
    T, dt, tau, u, v0 = 12, 0.05, 0.3, 1.8, 1.0
    sc = S.scenario("small", K=1, T=T, N=4, O=0, path="straight", sigma=(0.0, 0.0))
    sc = sc.replace(Y=np.zeros_like(sc.Y), x0=np.array([2.0, 0.0, 0.0, v0, 0.0]))
    goal = (2.5, 0.0)
    P0 = sc.params
    P1 = sc.params.__class__(**{**P0.__dict__, "beta": (0.0, 1.0, 0.7, 0.4), "goal": goal,
                                "goal_radius": 0.2, "P_goal": 50.0})
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = np.tile([u, 0.0], (T, 1))
    base = O.rollout(sc, fits, sc.x0, U, 0)["stage"][0]
    withg = O.rollout(sc.replace(params=P1), fits, sc.x0, U, 0)["stage"][0]
    X, v = 2.0, v0
    expect = []
    for k in range(T):
        X, v = X + dt * v, v + dt / tau * (u - v)
        d = abs(X - goal[0])
        e = 0.7 * d
        if k == T - 1:
            e += 0.4 * 50.0 * (1.0 if d > 0.2 else 0.0)
        expect.append(e)
    np.testing.assert_allclose(withg - base, expect, rtol=1e-12, atol=1e-12)
    # the terminal indicator fires in this case (the robot overshoots the goal)
    assert abs(X - goal[0]) > 0.2


def _qp_data(seed, H=25, M=3):
    rng = np.random.default_rng(seed)
    Fv = rng.normal(size=(H, M))
    Fw = rng.normal(size=(H, M))
    return rng, Fv, Fw


def test_terrain_weights_exact_recovery():
    rng, Fv, Fw = _qp_data(1)
    w_true = np.array([0.2, 0.5, 0.3])
    w = O.terrain_weights(Fv @ w_true, Fw @ w_true, Fv, Fw, np.full(3, 1 / 3), 0.0)
    np.testing.assert_allclose(w, w_true, atol=1e-7)


def test_terrain_weights_equality_constrained_least_squares():
    """gamma = 0 with an interior minimiser: the KKT system of least squares on sum w = 1."""
    rng, Fv, Fw = _qp_data(2)
    w_true = np.array([0.3, 0.3, 0.4])
    Yv = Fv @ w_true + 0.05 * rng.normal(size=Fv.shape[0])
    Yw = Fw @ w_true + 0.05 * rng.normal(size=Fw.shape[0])
    Q = Fv.T @ Fv + Fw.T @ Fw
    c = Fv.T @ Yv + Fw.T @ Yw
    A = np.block([[2 * Q, np.ones((3, 1))], [np.ones((1, 3)), np.zeros((1, 1))]])
    sol = np.linalg.solve(A, np.r_[2 * c, 1.0])[:3]
    assert np.all(sol > 0.01)
    w = O.terrain_weights(Yv, Yw, Fv, Fw, np.full(3, 1 / 3), 0.0)
    np.testing.assert_allclose(w, sol, atol=1e-7)


def test_terrain_weights_large_gamma_keeps_previous():
    rng, Fv, Fw = _qp_data(3)
    Yv, Yw = rng.normal(size=25), rng.normal(size=25)
    w_prev = np.array([0.6, 0.1, 0.3])
    w = O.terrain_weights(Yv, Yw, Fv, Fw, w_prev, 1e6)
    np.testing.assert_allclose(w, w_prev, atol=1e-9)


@pytest.mark.parametrize("seed,gamma", [(4, 0.0), (5, 0.5), (6, 3.0), (7, 20.0)])
def test_terrain_weights_brute_force(seed, gamma):
    rng, Fv, Fw = _qp_data(seed, H=15)
    Yv, Yw = rng.normal(size=15), rng.normal(size=15)
    w_prev = rng.dirichlet(np.ones(3))
    w = O.terrain_weights(Yv, Yw, Fv, Fw, w_prev, gamma)
    assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-12
    best = O.terrain_objective(w, Yv, Yw, Fv, Fw, w_prev, gamma)
    n = 400
    grid_best, grid_w = np.inf, None
    for i, j in itertools.product(range(n + 1), range(n + 1)):
        if i + j > n:
            continue
        g = np.array([i, j, n - i - j]) / n
        val = O.terrain_objective(g, Yv, Yw, Fv, Fw, w_prev, gamma)
        if val < grid_best:
            grid_best, grid_w = val, g
    assert best <= grid_best + 1e-12
    assert np.max(np.abs(w - grid_w)) < 0.02
