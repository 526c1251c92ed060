"""GPU parity: Philox draws, control noise, GP fit factors and GP posterior."""
import numpy as np
import pytest

import oracle as O
import scenarios as S

pytestmark = pytest.mark.gpu


def test_philox_bit_exact(lib):
    import torch
    rng = np.random.default_rng(0)
    M = 1 << 20
    ctr = rng.integers(0, 2**32, size=(M, 4), dtype=np.uint64)
    ctr[:16] = 0
    ctr[16:32, 2:] = 0xFFFFFFFF          # high counter words (iteration) set
    for seed in (0, 1, 0xDEADBEEFCAFEBABE, 2**64 - 1):
        c_d = torch.tensor(ctr.astype(np.uint32).view(np.int32), device="cuda")
        out = torch.empty_like(c_d)
        lib.gpmppi_philox(seed, c_d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        ref = O.philox4x32_10(ctr, O.philox.seed_key(seed))
        assert np.array_equal(got, ref)


def test_control_noise_matches_oracle(lib):
    import torch
    K, T = 3000, 37
    sigma = (0.5, 0.8)
    for it in (0, 5, (1 << 32) + 3):
        eps = torch.empty(K, T, 2, device="cuda")
        lib.gpmppi_control_noise(123456789, K, T, it, sigma, eps)
        torch.cuda.synchronize()
        got = eps.cpu().numpy().astype(np.float64)
        ref = np.stack([O.control_noise(123456789, k, np.arange(K), it, sigma) for k in range(T)], axis=1)
        # FP32 Box-Muller: relative error of a few ulp in the radius and angle
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("N", [1, 45, 500, 1000])
def test_gp_fit_factors_fp64(lib, N):
    sc = S.scenario("cfg2", N=N)
    g = lib.gp_fit(sc.X, sc.Y, sc.hyper)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    for j in range(2):
        Linv, alpha = lib.gp_factors(g, j)
        ref = fits[j]
        scale = np.max(np.abs(ref["Linv"]))
        assert np.max(np.abs(Linv - ref["Linv"])) <= 1e-10 * scale
        assert np.max(np.abs(alpha - ref["alpha"])) <= 1e-8 * max(1.0, np.max(np.abs(ref["alpha"])))
        assert np.all(np.triu(Linv, 1) == 0.0)


def test_gp_fit_not_pd(lib):
    X = np.tile(np.array([[0.5, 0.1, 1.0, 0.2]]), (4, 1))      # identical inputs
    h = S.Hyper(noise_var=0.0)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.gp_fit(X, np.zeros((4, 2)), (h, h))
    assert ei.value.code == lib.GPMPPI_ERR_NOT_PD


@pytest.mark.parametrize("N,distinct", [(45, False), (500, False), (333, True), (0, False)])
def test_gp_predict(lib, N, distinct):
    import torch
    sc = S.scenario("cfg2", N=N)
    hyper = sc.hyper
    if distinct:
        hyper = (S.Hyper(lengthscale=(0.5, 0.6, 0.7, 0.8), signal_var=0.1, noise_var=1e-4),
                 S.Hyper(lengthscale=(0.9, 0.4, 0.5, 0.6), signal_var=0.05, noise_var=2e-4))
    g = lib.gp_fit(sc.X, sc.Y, hyper)
    rng = np.random.default_rng(3)
    Z = S.GP_INPUT_LO + (S.GP_INPUT_HI - S.GP_INPUT_LO) * rng.random((700, 4))
    Z[:5] = sc.X[:5] if N >= 5 else Z[:5]
    Zd = torch.tensor(Z, dtype=torch.float32, device="cuda")
    mean = torch.empty(700, 2, device="cuda")
    var = torch.empty(700, 2, device="cuda")
    lib.gp_predict(g, Zd, mean, var)
    torch.cuda.synchronize()
    fits = O.gp_fit(sc.X, sc.Y, hyper)
    m_ref, v_ref = O.gp_predict(fits, Z.astype(np.float32).astype(np.float64))
    sf2 = np.array([hyper[0].signal_var, hyper[1].signal_var])
    assert np.max(np.abs(mean.cpu().numpy() - m_ref)) <= 2e-5
    assert np.all(np.abs(var.cpu().numpy() - v_ref) <= 1e-4 * sf2)
    assert np.all(var.cpu().numpy() >= 0) and np.all(var.cpu().numpy() <= sf2 * (1 + 1e-6))
