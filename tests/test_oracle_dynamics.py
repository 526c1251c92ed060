"""Pins for the oracle's motion model (Eq. 1-2, Eq. 6) and covariance (Eq. 10).

Closed forms: with zero GP residual and no sampling noise the first-order
lag gives v(k) = v_c + (v0 - v_c) a^k, a = 1 - dt/tau_v, and positions are
geometric sums; at steady (v, omega) the path is a circular arc with the
chord-sum closed form.  The Jacobian is pinned by central finite differences
of the nominal step, and the covariance recursion by the matrix-power sum of
a time-invariant linear system.
"""
import numpy as np
import pytest

import oracle as O
import scenarios as S


def lab(K=3, T=30, sf2=1e-30, far=False, noise=(0.0, 0.0), **kw):
    """A tiny scenario with a residual-free GP (targets 0) and no sampling noise.

    far=True puts the training set far away so the GP variance equals sf2
    exactly; sf2 tiny makes the variance vanish."""
    sc = S.scenario("small", K=K, T=T, O=0, **kw)
    X = np.full((3, 4), 100.0) if far else S.GP_INPUT_LO + 0.5 * (S.GP_INPUT_HI - S.GP_INPUT_LO) * np.ones((3, 4))
    X = X + np.arange(3)[:, None] * 0.1
    h = S.Hyper(lengthscale=(0.5,) * 4, signal_var=sf2, noise_var=1e-4)
    sc = sc.replace(X=X, Y=np.zeros((3, 2)), hyper=(h, h), obstacles=np.zeros((0, 3)))
    sc.params.sigma = noise
    return sc


def run(sc, x0, U):
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    return O.rollout(sc, fits, x0, U, it=0)


def test_straight_line_closed_form():
    sc = lab(T=40)
    P = sc.params
    th0, v0, vc = 0.37, 0.4, 1.7
    x0 = np.array([1.0, -2.0, th0, v0, 0.0])
    U = np.tile([vc, 0.0], (P.T, 1))
    ro = run(sc, x0, U)
    a = 1.0 - P.dt / P.tau_v
    k = np.arange(P.T + 1)
    v = vc + (v0 - vc) * a ** k                      # v(0) .. v(T)
    csum = np.concatenate([[0.0], np.cumsum(v[:-1])])  # sum_{j<k} v(j)
    X = x0[0] + P.dt * np.cos(th0) * csum
    Y = x0[1] + P.dt * np.sin(th0) * csum
    mu = ro["mu"][0]                                 # states after steps 1..T
    np.testing.assert_allclose(mu[:, 3], v[1:], rtol=1e-13)
    np.testing.assert_allclose(mu[:, 0], X[1:], rtol=1e-12)
    np.testing.assert_allclose(mu[:, 1], Y[1:], rtol=1e-12)
    np.testing.assert_allclose(mu[:, 2], th0, rtol=0, atol=0)
    np.testing.assert_allclose(mu[:, 4], 0.0, atol=0)


def test_constant_arc_closed_form():
    sc = lab(T=60)
    P = sc.params
    th0, v, w = -0.8, 1.2, 0.9
    x0 = np.array([0.5, 0.25, th0, v, w])
    U = np.tile([v, w], (P.T, 1))
    mu = run(sc, x0, U)["mu"][0]
    phi = P.dt * w
    k = np.arange(1, P.T + 1)
    chord = P.dt * v * np.sin(k * phi / 2) / np.sin(phi / 2)
    mid = th0 + (k - 1) * phi / 2
    np.testing.assert_allclose(mu[:, 2], th0 + k * phi, rtol=1e-13)
    np.testing.assert_allclose(mu[:, 0], x0[0] + chord * np.cos(mid), rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(mu[:, 1], x0[1] + chord * np.sin(mid), rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(mu[:, 3], v, rtol=1e-15)
    np.testing.assert_allclose(mu[:, 4], w, rtol=1e-15)


def test_jacobian_finite_differences():
    rng = np.random.default_rng(4)
    P = S.Params()
    for _ in range(20):
        mu = rng.standard_normal(5)
        u = rng.standard_normal(2)
        A = O.jacobian(mu, P.dt, P.tau_v, P.tau_w)
        h = 1e-6
        for i in range(5):
            e = np.zeros(5)
            e[i] = h
            col = (O.nominal_step(mu + e, u, P.dt, P.tau_v, P.tau_w)
                   - O.nominal_step(mu - e, u, P.dt, P.tau_v, P.tau_w)) / (2 * h)
            np.testing.assert_allclose(A[:, i], col, atol=1e-8)


def test_covariance_matches_matrix_power_sum():
    sf2 = 0.07
    sc = lab(T=25, sf2=sf2, far=True)
    P = sc.params
    v = 1.3
    x0 = np.array([0.0, 0.0, 0.0, v, 0.0])
    U = np.tile([v, 0.0], (P.T, 1))
    ro = run(sc, x0, U)
    np.testing.assert_allclose(ro["var"][0], sf2, rtol=0, atol=0)
    # the state stays at theta = omega = 0 and v = v_c, so the linearisation is
    # time invariant; take it from finite differences of the nominal step
    A = np.zeros((5, 5))
    h = 1e-6
    for i in range(5):
        e = np.zeros(5)
        e[i] = h
        A[:, i] = (O.nominal_step(x0 + e, U[0], P.dt, P.tau_v, P.tau_w)
                   - O.nominal_step(x0 - e, U[0], P.dt, P.tau_v, P.tau_w)) / (2 * h)
    Q = np.diag([0, 0, 0, sf2, sf2])
    for k in range(1, P.T + 1):
        ref = sum(np.linalg.matrix_power(A, j) @ Q @ np.linalg.matrix_power(A, j).T for j in range(k))
        np.testing.assert_allclose(ro["Sigma"][0, k - 1], ref, rtol=1e-7, atol=1e-14)


def test_zero_variance_keeps_covariance_zero():
    sc = lab(T=15, sf2=1e-300)
    x0 = np.array([0.0, 0.0, 0.2, 1.0, 0.3])
    ro = run(sc, x0, np.tile([1.0, 0.3], (15, 1)))
    assert np.max(np.abs(ro["Sigma"])) < 1e-290


def test_covariance_symmetric_psd_on_noisy_rollout():
    sc = S.scenario("small")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, it=3)
    Sg = ro["Sigma"]
    np.testing.assert_allclose(Sg, np.swapaxes(Sg, -1, -2), atol=1e-15)
    ev = np.linalg.eigvalsh(Sg)
    assert np.all(ev > -1e-12)
    assert np.all(ro["var"] >= 0) and np.all(ro["var"] <= sc.hyper[0].signal_var)


def test_zero_residual_reduces_to_nominal_model():
    # targets 0 -> alpha = 0 -> GP mean 0: rollout equals iterating nominal_step
    sc = lab(T=12, noise=(0.5, 0.8))
    sc.params.K = 5
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    x0 = np.array([0.0, 0.0, 0.1, 1.0, 0.0])
    U = np.tile([1.5, 0.2], (12, 1))
    ro = O.rollout(sc, fits, x0, U, it=0)
    mu = np.tile(x0, (5, 1))
    for k in range(12):
        mu = O.nominal_step(mu, ro["u_tilde"][:, k], sc.params.dt, sc.params.tau_v, sc.params.tau_w)
        np.testing.assert_allclose(ro["mu"][:, k], mu, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_gp_query_composition(d):
    # One training point and an ARD kernel that only sees input d: the GP mean
    # of the first step has the N = 1 closed form evaluated at component d of
    # z = (v(0), omega(0), u~_v(0), u~_omega(0)); distinct values per component
    # make any index mix-up fail.
    sc = lab(T=1)
    P = sc.params
    ell = [1e6] * 4
    ell[d] = 0.4
    h = S.Hyper(lengthscale=tuple(ell), signal_var=0.2, noise_var=0.05)
    xt = np.array([[0.9, 0.2, 1.1, -0.4]])
    yt = np.array([[0.3, -0.5]])
    sc = sc.replace(X=xt, Y=yt, hyper=(h, h))
    x0 = np.array([0.0, 0.0, 0.0, 1.4, -0.7])       # v(0) = 1.4, omega(0) = -0.7
    U = np.array([[0.6, 0.9]])                       # inside the box: no clamping
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    mu1 = O.rollout(sc, fits, x0, U, it=0)["mu"][0, 0]
    z = np.array([1.4, -0.7, 0.6, 0.9])
    k = 0.2 * np.exp(-0.5 * ((z[d] - xt[0, d]) / 0.4) ** 2) * np.exp(
        -0.5 * np.sum(np.delete((z - xt[0]) / 1e6, d) ** 2))
    m = k * yt[0] / (0.2 + 0.05)
    nom = O.nominal_step(x0, U[0], P.dt, P.tau_v, P.tau_w)
    np.testing.assert_allclose(mu1[3], nom[3] + m[0], rtol=1e-13)
    np.testing.assert_allclose(mu1[4], nom[4] + m[1], rtol=1e-13)
