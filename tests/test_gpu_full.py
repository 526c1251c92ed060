"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times.

cfg2 (K=4096, T=50, N=500) is compared in full: every sample's cost, the
weights and U_new.  For the larger shapes the oracle recomputes a sample of
rows one by one (samples are independent given U and the Philox key), and the
update is checked through properties that hold at any size."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from parity import (TOL_U, check_step, check_trace, gpu_step, gpu_trace, make_ctrl,
                    reconcile_costs, assert_close, TOL_COST)

pytestmark = pytest.mark.gpu


def _rows(K, mt_guess=27, n=48, seed=0):
    rng = np.random.default_rng(seed)
    rows = {0, 1, K - 1, K - 2, mt_guess - 1, mt_guess, 2 * mt_guess}
    rows |= set(rng.integers(0, K, n).tolist())
    return np.array(sorted(r for r in rows if 0 <= r < K))


def _noise_controls(sc, U, it):
    """u~ for every sample from the oracle's noise (FP64), (K, T, 2)."""
    P = sc.params
    ut = np.empty((P.K, P.T, 2))
    for k in range(P.T):
        eps = O.control_noise(P.seed, k, np.arange(P.K), it, P.sigma)
        ut[:, k] = np.clip(U[k] + eps, P.u_min, P.u_max)
    return ut


def test_cfg2_full_step(lib):
    sc = S.scenario("cfg2")
    g, ctrl = make_ctrl(lib, sc)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 0)
    info = check_step(sc, ro, sc.U0, U_new, w, c)
    print("cfg2 full step", info)
    assert info["n_alt"] <= 0.01 * sc.params.K


def test_cfg2_sampled_trajectories(lib):
    sc = S.scenario("cfg2")
    g, ctrl = make_ctrl(lib, sc)
    U = sc.U0.copy()
    U[:, 1] = 0.4 * np.sin(np.linspace(0, 3, sc.params.T))
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=3)
    rows = _rows(sc.params.K)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, U, 3, samples=rows)
    info = check_trace(sc, ro, tr, rows)
    ref_c, n_alt = reconcile_costs(sc, ro, tr["costs"][rows], rows)
    assert_close(tr["costs"][rows], ref_c, TOL_COST, what="costs")
    print("cfg2 sampled", info, n_alt)


@pytest.mark.parametrize("name", ["cfg4", "cfg3"])
def test_large_shapes_sampled_and_properties(lib, name):
    import torch
    sc = S.scenario(name, precision=0)       # the FP32 CUDA-core path
    P = sc.params
    g, ctrl = make_ctrl(lib, sc)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    rows = _rows(P.K, n=24)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 1, samples=rows)
    check_trace(sc, ro, tr, rows)
    ref_c, _ = reconcile_costs(sc, ro, tr["costs"][rows], rows)
    assert_close(tr["costs"][rows], ref_c, TOL_COST, what="costs")
    # full step: weights are the softmax of the costs, U_new the weighted sum
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    np.testing.assert_allclose(c, tr["costs"], rtol=1e-6, atol=1e-6)
    w_from_c = O.mppi_weights(c, P.lam)
    assert np.max(np.abs(w - w_from_c)) <= 1e-5
    assert abs(w.sum() - 1.0) <= 1e-5
    ut = _noise_controls(sc, sc.U0, 1)
    U_chk = sc.U0 + np.einsum("s,skc->kc", w, ut - sc.U0[None])
    assert np.max(np.abs(U_new - U_chk)) <= TOL_U
    assert np.all(U_new[:, 0] >= P.u_min[0] - 1e-6) and np.all(U_new[:, 0] <= P.u_max[0] + 1e-6)
    del torch
