"""Terrain ensemble (Eq. 3) and goal terms (Eq. 12) on the GPU against the
FP64 oracle: full steps and per-step traces on small cases, sampled rows of
the 4096-sample workload with three terrains, weight updates (Eq. 4) fed
back into the rollout, the goal terms on every rollout path and in the
adjoint, and the combinations the library rejects."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from parity import (TOL_COST, TOL_U, assert_close, check_step, check_trace, gpu_step, gpu_trace,
                    make_ctrl, reconcile_costs, to_np)

pytestmark = pytest.mark.gpu


def _x0(sc):
    return sc.x0.astype(np.float32).astype(np.float64)


def _U(sc, seed=0):
    U = sc.U0.copy()
    U[:, 1] = 0.5 * np.sin(np.arange(sc.params.T) + seed)
    return U


@pytest.mark.parametrize("M", [2, 3, 5])
def test_ensemble_small_full_step_and_trace(lib, M):
    sc = S.terrain_scenario("small", M=M, N=40)
    gps, ctrl = make_ctrl(lib, sc)
    U = _U(sc)
    ens = O.fit_scenario(sc)
    ro = O.rollout(sc, ens, _x0(sc), U, 0)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=0)
    info_t = check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=0)
    info = check_step(sc, ro, U, U_new, w, c)
    print(M, info_t, info)


@pytest.mark.parametrize("precision,M,N", [(2, 2, 40), (2, 3, 300), (3, 3, 40), (2, 2, 800), (1, 2, 200)])
def test_ensemble_split_precision_full_step_and_trace(lib, precision, M, N):
    """The ensemble on the tensor cores: the GPs' factors stacked block-diagonally
    through the streaming rollout (odd block counts padded, the second column
    set beyond 768 points, the three-term BF16 split)."""
    sc = S.terrain_scenario("small", M=M, N=N, precision=precision)
    gps, ctrl = make_ctrl(lib, sc)
    assert lib.mppi_rollout_kind(ctrl) == lib.GPMPPI_KERNEL_TC_STREAM
    U = _U(sc)
    ens = O.fit_scenario(sc)
    ro = O.rollout(sc, ens, _x0(sc), U, 0)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=0)
    info_t = check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=0)
    info = check_step(sc, ro, U, U_new, w, c)
    np.testing.assert_allclose(tr["costs"], c, rtol=1e-6, atol=1e-6)
    print(precision, M, N, info_t, info)


def test_ensemble_split_weight_change_and_fp32_agreement(lib):
    """New weights reach the tensor-core ensemble at the next step, and its
    costs agree with the FP32 ensemble's."""
    sc2 = S.terrain_scenario("small", M=3, N=60, precision=2)
    sc0 = S.terrain_scenario("small", M=3, N=60, precision=0)
    _, c2 = make_ctrl(lib, sc2)
    _, c0 = make_ctrl(lib, sc0)
    U = _U(sc2, 3)
    for w in (None, (0.2, 0.5, 0.3)):
        if w is not None:
            lib.mppi_set_terrain_weights(c2, w)
            lib.mppi_set_terrain_weights(c0, w)
            sc2 = sc2.replace(terrain_w=tuple(float(x) for x in np.float32(w)))
        Ua, wa, ca = gpu_step(lib, c2, sc2, sc2.x0, U, it=6)
        Ub, wb, cb = gpu_step(lib, c0, sc0, sc0.x0, U, it=6)
        np.testing.assert_allclose(ca, cb, rtol=2e-5, atol=2e-5)
        assert np.max(np.abs(Ua - Ub)) <= TOL_U
        ro = O.rollout(sc2, O.fit_scenario(sc2), _x0(sc2), U, 6)
        check_step(sc2, ro, U, Ua, wa, ca)


def test_ensemble_one_hot_equals_single_gp(lib):
    import torch
    sc = S.terrain_scenario("small", M=3, N=40, w=(0.0, 1.0, 0.0))
    gps, ctrl = make_ctrl(lib, sc)
    X, Y, h = sc.terrains[1]
    single = sc.replace(X=X, Y=Y, hyper=h, terrains=None, terrain_w=None)
    _, c1 = make_ctrl(lib, single)
    U = _U(sc)
    Ua, wa, ca = gpu_step(lib, ctrl, sc, sc.x0, U, it=3)
    Ub, wb, cb = gpu_step(lib, c1, single, sc.x0, U, it=3)
    np.testing.assert_allclose(ca, cb, rtol=2e-5, atol=2e-5)
    assert np.max(np.abs(Ua - Ub)) <= TOL_U
    del torch


def test_ensemble_weight_update_loop(lib):
    """Alg. 1 Step 3: predictions of each terrain at observed inputs (gp_predict
    on the device), weights from the library's exact Eq. 4 solver, fed back
    with mppi_set_terrain_weights; the next step matches the oracle with them."""
    import torch
    sc = S.terrain_scenario("small", M=3, N=40)
    gps, ctrl = make_ctrl(lib, sc)
    rng = np.random.default_rng(5)
    H = 12
    Z = rng.uniform(S.GP_INPUT_LO, S.GP_INPUT_HI, (H, 4))
    truth = S.terrain_residual(0, Z[:, 0], Z[:, 1], Z[:, 2], Z[:, 3])      # the robot is on terrain 0
    Fv, Fw = np.zeros((H, 3)), np.zeros((H, 3))
    Zd = torch.tensor(Z, dtype=torch.float32, device="cuda")
    for i, g in enumerate(gps):
        m = torch.empty(H, 2, device="cuda")
        v = torch.empty(H, 2, device="cuda")
        lib.gp_predict(g, Zd, m, v)
        torch.cuda.synchronize()
        Fv[:, i], Fw[:, i] = to_np(m)[:, 0], to_np(m)[:, 1]
    w_prev = np.array(sc.terrain_w)
    w = lib.terrain_weights(truth[:, 0], truth[:, 1], Fv, Fw, w_prev, 1e-3)
    wo = O.terrain_weights(truth[:, 0], truth[:, 1], Fv, Fw, w_prev, 1e-3)
    np.testing.assert_allclose(w, wo, atol=2e-4)
    assert np.argmax(w) == 0                # the estimate puts most weight on the true terrain
    lib.mppi_set_terrain_weights(ctrl, w)
    sc2 = sc.replace(terrain_w=tuple(float(x) for x in np.float32(w)))
    U = _U(sc, 1)
    ro = O.rollout(sc2, O.fit_scenario(sc2), _x0(sc2), U, 4)
    U_new, wt, c = gpu_step(lib, ctrl, sc2, sc.x0, U, it=4)
    check_step(sc2, ro, U, U_new, wt, c)


@pytest.mark.parametrize("precision", [0, 2])
def test_ensemble_cfg2_three_terrains_sampled(lib, precision):
    """K=4096, T=50, three terrains of N=500: sampled rows recomputed by the oracle."""
    sc = S.terrain_scenario("cfg2", M=3, precision=precision)
    P = sc.params
    gps, ctrl = make_ctrl(lib, sc)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    rng = np.random.default_rng(2)
    rows = np.array(sorted({0, 7, 8, P.K - 1} | set(rng.integers(0, P.K, 20).tolist())))
    ro = O.rollout(sc, O.fit_scenario(sc), _x0(sc), sc.U0, 1, samples=rows)
    info = check_trace(sc, ro, tr, rows)
    ref_c, _ = reconcile_costs(sc, ro, tr["costs"][rows], rows)
    assert_close(tr["costs"][rows], ref_c, TOL_COST, what="costs")
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    np.testing.assert_allclose(c, tr["costs"], rtol=1e-6, atol=1e-6)
    assert abs(w.sum() - 1.0) <= 1e-5
    print("cfg2 terrain3 precision", precision, info)


def _goal_scenario(precision=0, **kw):
    sc = S.scenario("small", precision=precision, **kw)
    P = sc.params
    # goal near where the 7-step rollouts end (about (0.28, 0.28), spread 1.5 cm):
    # the terminal term fires for some samples and not for others
    P2 = P.__class__(**{**P.__dict__, "beta": (0.0, 1.0, 0.4, 0.6), "goal": (0.28, 0.28),
                        "goal_radius": 0.02, "P_goal": 80.0})
    return sc.replace(params=P2)


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_goal_terms_all_paths(lib, precision):
    sc = _goal_scenario(precision)
    _, ctrl = make_ctrl(lib, sc)
    U = _U(sc, 2)
    ro = O.rollout(sc, O.gp_fit(sc.X, sc.Y, sc.hyper), _x0(sc), U, 0)
    # the terminal term must fire for some samples and not for others
    T = sc.params.T
    dg = np.hypot(ro["mu"][:, T - 1, 0] - sc.params.goal[0], ro["mu"][:, T - 1, 1] - sc.params.goal[1])
    assert 0 < np.sum(dg > sc.params.goal_radius) < sc.params.K
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=0)
    check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=0)
    check_step(sc, ro, U, U_new, w, c)


def test_goal_terms_ensemble(lib):
    sc = S.terrain_scenario("small", M=3, N=40)
    P = sc.params
    P2 = P.__class__(**{**P.__dict__, "beta": (0.0, 1.0, 0.4, 0.6), "goal": (0.28, 0.28),
                        "goal_radius": 0.02, "P_goal": 80.0})
    sc = sc.replace(params=P2)
    gps, ctrl = make_ctrl(lib, sc)
    U = _U(sc, 2)
    ro = O.rollout(sc, O.fit_scenario(sc), _x0(sc), U, 0)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=0)
    check_step(sc, ro, U, U_new, w, c)


def test_goal_terms_gradient(lib):
    """The adjoint with the goal terms (F smoothed by the same sigmoid) against
    the oracle's FP64 gradient."""
    import torch
    sc = _goal_scenario(0)
    _, ctrl = make_ctrl(lib, sc)
    U = _U(sc, 2)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    J, dU, dl = lib.mppi_grad(ctrl, sc.x0, Ud, 20.0)
    torch.cuda.synchronize()
    gU, gL = O.fd_gradient(sc, sc.hyper, _x0(sc), U.astype(np.float32).astype(np.float64), 0, None, 20.0)
    Jo, _ = O.objective(sc, sc.hyper, _x0(sc), U.astype(np.float32).astype(np.float64), 0, None, 20.0)
    assert abs(float(to_np(J)[0]) - Jo) <= 1e-4 * abs(Jo)
    for g, ref in ((to_np(dU), gU), (to_np(dl), gL)):
        floor = 1e-3 * np.max(np.abs(ref))      # the gradient tests' reading (test_gpu_grad.grad_err)
        assert np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor)) <= 1e-3


def test_ensemble_rejections(lib):
    import torch
    sc = S.terrain_scenario("small", M=2, N=20)
    gps = [lib.gp_fit(X, Y, h) for X, Y, h in sc.terrains]
    P = sc.params
    for field, val in (("variance_mode", 1),):
        P2 = P.__class__(**{**P.__dict__, field: val})
        with pytest.raises(lib.GpmppiError) as ei:
            lib.mppi_create_ensemble(P2, sc.obstacles, sc.path, gps, sc.terrain_w)
        assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED
    ctrl = lib.mppi_create_ensemble(P, sc.obstacles, sc.path, gps, sc.terrain_w)
    U = torch.tensor(sc.U0, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_grad(ctrl, sc.x0, U, 20.0)
    assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_batch_create([ctrl])
    assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_set_terrain_weights(ctrl, [1.0, 0.0, 0.0])
    assert ei.value.code == lib.GPMPPI_ERR_INVALID_ARG
    # the GPs stay referenced by the controller
    with pytest.raises(lib.GpmppiError):
        lib.gp_destroy(gps[1])
    lib.mppi_destroy(ctrl)
    lib.gp_destroy(gps[1])
