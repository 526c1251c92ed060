"""Pins for the oracle's GP fit / predict (Sec. III-A, Eq. 3)."""
import os

import numpy as np
import pytest

import oracle as O
import scenarios as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hyper(ell=0.5, sf2=0.1, sn2=1e-4):
    return S.Hyper(lengthscale=(ell,) * 4, signal_var=sf2, noise_var=sn2)


def test_single_point_closed_form():
    # N = 1: m = k y / (sf2 + sn2), var = sf2 - k^2 / (sf2 + sn2)
    h = S.Hyper(lengthscale=(0.5, 0.7, 0.9, 1.3), signal_var=0.3, noise_var=0.02)
    x = np.array([[0.3, -0.2, 1.1, 0.4]])
    y = np.array([[0.25, -0.6]])
    fits = O.gp_fit(x, y, (h, h))
    z = np.array([[0.5, 0.1, 0.9, 0.2], [0.3, -0.2, 1.1, 0.4]])
    m, v = O.gp_predict(fits, z)
    for i in range(z.shape[0]):
        r2 = np.sum(((z[i] - x[0]) / np.array(h.lengthscale)) ** 2)
        k = h.signal_var * np.exp(-0.5 * r2)
        den = h.signal_var + h.noise_var
        np.testing.assert_allclose(m[i], k * y[0] / den, rtol=1e-13)
        np.testing.assert_allclose(v[i], h.signal_var - k * k / den, rtol=1e-13)


def test_far_field_reverts_to_prior():
    rng = np.random.default_rng(0)
    X = rng.random((40, 4))
    Y = rng.standard_normal((40, 2))
    fits = O.gp_fit(X, Y, (_hyper(), _hyper()))
    m, v = O.gp_predict(fits, np.full((3, 4), 50.0))
    assert np.all(np.abs(m) < 1e-300 + 1e-12)
    np.testing.assert_allclose(v, 0.1, rtol=0, atol=1e-15)


def test_variance_bounds_and_interpolation():
    sc = S.scenario("cfg1")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    rng = np.random.default_rng(1)
    Z = S.GP_INPUT_LO + (S.GP_INPUT_HI - S.GP_INPUT_LO) * rng.random((500, 4))
    m, v = O.gp_predict(fits, Z)
    assert np.all(v >= 0.0) and np.all(v <= 0.1)
    # at the training inputs the posterior mean is close to the targets and
    # the variance is of the order of the noise variance
    m, v = O.gp_predict(fits, sc.X)
    assert np.max(np.abs(m - sc.Y)) < 0.05
    assert np.max(v) < 1e-3


def test_against_sklearn():
    sk = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    sc = S.scenario("cfg1")
    ell = np.array([0.5, 0.6, 0.7, 0.8])
    h = S.Hyper(lengthscale=tuple(ell), signal_var=0.1, noise_var=1e-4)
    fits = O.gp_fit(sc.X, sc.Y, (h, h))
    rng = np.random.default_rng(2)
    Z = S.GP_INPUT_LO + (S.GP_INPUT_HI - S.GP_INPUT_LO) * rng.random((200, 4))
    m, v = O.gp_predict(fits, Z)
    for j in range(2):
        gpr = sk.GaussianProcessRegressor(
            kernel=kern.ConstantKernel(0.1, "fixed") * kern.RBF(ell, "fixed"),
            alpha=1e-4, optimizer=None, normalize_y=False)
        gpr.fit(sc.X, sc.Y[:, j])
        mm, sd = gpr.predict(Z, return_std=True)
        np.testing.assert_allclose(m[:, j], mm, rtol=1e-7, atol=1e-10)
        np.testing.assert_allclose(v[:, j], sd ** 2, rtol=1e-6, atol=1e-10)


def test_factor_identities():
    sc = S.scenario("small")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    f = fits[0]
    Kxx = O.se_ard(sc.X, sc.X, f["lengthscale"], f["signal_var"]) + f["noise_var"] * np.eye(sc.N)
    np.testing.assert_allclose(f["L"] @ f["L"].T, Kxx, atol=1e-14)
    np.testing.assert_allclose(f["Linv"] @ f["L"], np.eye(sc.N), atol=1e-9)
    np.testing.assert_allclose(Kxx @ f["alpha"], sc.Y[:, 0], atol=1e-10)


def test_tightening_constants_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "tightening_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    p = vals["p_x"]
    assert O.chi2_2_quantile(p) == pytest.approx(vals["chi2_2"], rel=1e-15)
    assert np.sqrt(O.chi2_2_quantile(p)) == pytest.approx(vals["sqrt_chi2_2"], rel=1e-15)
    assert O.normal_quantile(p) == pytest.approx(vals["phi_inv"], rel=1e-14)


def test_quantiles_against_scipy():
    st = pytest.importorskip("scipy.stats")
    for p in (0.5, 0.8, 0.9, 0.95, 0.99, 0.999, 0.999999):
        assert O.chi2_2_quantile(p) == pytest.approx(st.chi2.ppf(p, 2), rel=1e-12)
        assert O.normal_quantile(p) == pytest.approx(st.norm.ppf(p), rel=1e-12, abs=1e-15)
