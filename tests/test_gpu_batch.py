"""Batched iterations of many independent controllers (uneven K, T, N,
obstacles, paths and precisions) against the FP64 oracle, against individual
mppi_step calls, through CUDA-graph replay and after autotuning."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from parity import TOL_U, check_step, make_ctrl, to_np

pytestmark = pytest.mark.gpu

SPECS = [  # (K, T, N, O, path, precision, seed)
    (300, 7, 200, 6, "eight", 2, 11),
    (77, 5, 45, 3, "sine", 2, 12),
    (513, 9, 333, 10, "straight", 2, 13),
    (129, 4, 0, 0, "eight", 2, 14),
    (260, 6, 140, 5, "sine", 1, 15),
    (200, 8, 90, 4, "eight", 0, 16),
    (190, 6, 260, 5, "sine", 3, 17),
]


def _scenarios():
    out = []
    for K, T, N, O_, path, prec, seed in SPECS:
        sc = S.scenario("small", K=K, T=T, N=N, O=O_, path=path, precision=prec, seed=seed)
        rng = np.random.default_rng(seed)
        x0 = sc.x0.copy()
        x0[3] = 0.5 + rng.random()
        U = np.tile([sc.params.v_desired, 0.0], (T, 1))
        U[:, 1] = 0.4 * np.sin(np.arange(T) + seed)
        out.append((sc, x0, U))
    return out


def _batch(lib):
    import torch
    items = _scenarios()
    ctrls = [make_ctrl(lib, sc)[1] for sc, _, _ in items]
    b = lib.mppi_batch_create(ctrls)
    for i, (sc, x0, U) in enumerate(items):
        b.state[i].copy_(torch.tensor(x0, dtype=torch.float32))
        b.U_nom[i].copy_(torch.tensor(U, dtype=torch.float32))
    return b, ctrls, items


def test_batch_matches_oracle_and_single_steps(lib):
    import torch
    b, ctrls, items = _batch(lib)
    lib.mppi_batch_step(b)
    torch.cuda.synchronize()
    for i, (sc, x0, U) in enumerate(items):
        fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
        ro = O.rollout(sc, fits, x0.astype(np.float32).astype(np.float64), U, 0)
        info = check_step(sc, ro, U, to_np(b.U_new[i]), to_np(b.weights[i]), to_np(b.costs[i]))
        assert lib.mppi_batch_get_iteration(b, i) == 1
        # the same controller stepped on its own
        Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
        U1 = torch.empty_like(Ud)
        w1 = torch.empty(sc.params.K, device="cuda")
        c1 = torch.empty_like(w1)
        lib.mppi_set_iteration(ctrls[i], 0)
        lib.mppi_step(ctrls[i], x0, Ud, U1, w1, c1)
        torch.cuda.synchronize()
        assert np.max(np.abs(to_np(U1) - to_np(b.U_new[i]))) <= TOL_U
        np.testing.assert_allclose(to_np(c1), to_np(b.costs[i]), rtol=1e-5, atol=1e-5)
        print(i, info)


def test_batch_graph_replay_equals_steps(lib):
    import torch
    b1, _, _ = _batch(lib)
    b2, _, _ = _batch(lib)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(3):
            lib.mppi_batch_step(b1, st)
            lib.mppi_batch_graph(b2, st)
    st.synchronize()
    for i in range(len(SPECS)):
        assert np.array_equal(to_np(b1.U_new[i]), to_np(b2.U_new[i]))
        assert np.array_equal(to_np(b1.costs[i]), to_np(b2.costs[i]))
        assert lib.mppi_batch_get_iteration(b2, i) == 3


def test_batch_autotune_keeps_parity(lib):
    import torch
    b, ctrls, items = _batch(lib)
    changed = lib.mppi_batch_autotune(b)
    assert 0 <= changed <= len(SPECS)
    for i, spec in enumerate(SPECS):
        rps, tile_us = lib.mppi_batch_layout(b, i)
        assert rps == (0 if spec[5] == 0 else rps) and (rps == 0 or rps in (2, 4, 8))
        assert tile_us > 0.0
    assert all(lib.mppi_batch_get_iteration(b, i) == 0 for i in range(len(SPECS)))
    lib.mppi_batch_step(b)
    torch.cuda.synchronize()
    for i, (sc, x0, U) in enumerate(items):
        fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
        ro = O.rollout(sc, fits, x0.astype(np.float32).astype(np.float64), U, 0)
        check_step(sc, ro, U, to_np(b.U_new[i]), to_np(b.weights[i]), to_np(b.costs[i]))


def test_batch_rejects_bad_groups(lib):
    sc = S.scenario("small")
    g, c = make_ctrl(lib, sc)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_batch_create([c, c])
    assert ei.value.code == lib.GPMPPI_ERR_INVALID_ARG
    sc2 = S.scenario("small", variance_mode=1)
    g2, c2 = make_ctrl(lib, sc2)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_batch_create([c, c2])
    assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED


def _cfg5_scenarios(B=64):
    """cfg5: 64 controllers, K 1024..16384, T 20..100, N 200..4096, 4..64
    obstacles, sinusoid / figure-eight paths; arithmetic cycling FP16 split,
    FP16 split, BF16 split, FP32."""
    scs = S.batched_scenarios(B)
    for i, sc in enumerate(scs):
        sc.params.precision = (2, 2, 1, 0)[i % 4]
    return scs


def test_batch_cfg5_shapes_sampled_rows_and_properties(lib):
    """The batched persistent launch at the cfg5 shapes, after autotuning:
    for every controller, the costs of sampled rows against the oracle's FP64
    rollout of those rows (indicator-tie protocol), the weights against the
    softmax of the controller's costs, and U_new against the weighted sum of
    the oracle's clamped sampled controls."""
    import torch
    from parity import TOL_COST, assert_close, reconcile_costs
    scs = _cfg5_scenarios()
    gps = [lib.gp_fit(sc.X, sc.Y, sc.hyper) for sc in scs]
    ctrls = [lib.mppi_create(sc.params, sc.obstacles, sc.path, g) for sc, g in zip(scs, gps)]
    b = lib.mppi_batch_create(ctrls)
    for i, sc in enumerate(scs):
        b.state[i].copy_(torch.tensor(sc.x0, dtype=torch.float32))
        b.U_nom[i].copy_(torch.tensor(sc.U0, dtype=torch.float32))
    lib.mppi_batch_autotune(b)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        lib.mppi_batch_graph(b, st)
    st.synchronize()
    rng = np.random.default_rng(5)
    layouts = []
    for i, sc in enumerate(scs):
        P = sc.params
        assert lib.mppi_batch_get_iteration(b, i) == 1
        c = to_np(b.costs[i])
        w = to_np(b.weights[i])
        U_new = to_np(b.U_new[i])
        rows = np.unique(np.concatenate([[0, P.K - 1], rng.integers(0, P.K, 2)]))
        fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
        ro = O.rollout(sc, fits, sc.x0.astype(np.float32).astype(np.float64), sc.U0, 0, samples=rows)
        ref_c, _ = reconcile_costs(sc, ro, c[rows], rows)
        assert_close(c[rows], ref_c, TOL_COST, what=f"controller {i} costs")
        assert np.max(np.abs(w - O.mppi_weights(c, P.lam))) <= 1e-5
        ut = np.empty((P.K, P.T, 2))
        for k in range(P.T):
            eps = O.control_noise(P.seed, k, np.arange(P.K), 0, P.sigma)
            ut[:, k] = np.clip(sc.U0[k] + eps, P.u_min, P.u_max)
        U_chk = sc.U0 + np.einsum("s,skc->kc", w, ut - sc.U0[None])
        assert np.max(np.abs(U_new - U_chk)) <= TOL_U, f"controller {i}"
        layouts.append(lib.mppi_batch_layout(b, i))
    print("cfg5 layouts (threads per sample, us per tile):", layouts)


def test_batch_with_terrain_ensembles(lib):
    """Terrain ensembles (Eq. 3) in the split precisions are items of the
    persistent launch: each matches its own mppi_step and the oracle, and a
    weight change on its controller reaches the next batched step, direct
    and graph-replayed."""
    import torch
    scs = [S.terrain_scenario("small", M=3, N=40, precision=2, K=150, T=6),
           S.terrain_scenario("small", M=2, N=300, precision=3, K=90, T=5),
           S.scenario("small", K=120, T=6, N=200, precision=2)]
    ctrls = [make_ctrl(lib, sc)[1] for sc in scs]
    b = lib.mppi_batch_create(ctrls)
    Us = []
    for i, sc in enumerate(scs):
        U = np.tile([sc.params.v_desired, 0.0], (sc.params.T, 1))
        U[:, 1] = 0.3 * np.sin(np.arange(sc.params.T) + i)
        Us.append(U)
        b.state[i].copy_(torch.tensor(sc.x0, dtype=torch.float32))
        b.U_nom[i].copy_(torch.tensor(U, dtype=torch.float32))

    def compare(it, oracle=False):
        for i, sc in enumerate(scs):
            Ud = torch.tensor(Us[i], dtype=torch.float32, device="cuda")
            U1 = torch.empty_like(Ud)
            w1 = torch.empty(sc.params.K, device="cuda")
            c1 = torch.empty_like(w1)
            lib.mppi_set_iteration(ctrls[i], it)
            lib.mppi_step(ctrls[i], sc.x0, Ud, U1, w1, c1)
            torch.cuda.synchronize()
            assert lib.mppi_batch_get_iteration(b, i) == it + 1
            assert np.max(np.abs(to_np(U1) - to_np(b.U_new[i]))) <= TOL_U
            np.testing.assert_allclose(to_np(c1), to_np(b.costs[i]), rtol=1e-5, atol=1e-5)
            if oracle:
                x0 = sc.x0.astype(np.float32).astype(np.float64)
                ro = O.rollout(sc, O.fit_scenario(sc), x0, Us[i], it)
                check_step(sc, ro, Us[i], to_np(b.U_new[i]), to_np(b.weights[i]), to_np(b.costs[i]))

    lib.mppi_batch_step(b)
    torch.cuda.synchronize()
    compare(0, oracle=True)
    lib.mppi_set_terrain_weights(ctrls[0], [0.1, 0.2, 0.7])
    scs[0] = scs[0].replace(terrain_w=tuple(float(x) for x in np.float32([0.1, 0.2, 0.7])))
    lib.mppi_batch_step(b)
    torch.cuda.synchronize()
    compare(1, oracle=True)
    lib.mppi_set_terrain_weights(ctrls[1], [0.6, 0.4])
    scs[1] = scs[1].replace(terrain_w=tuple(float(x) for x in np.float32([0.6, 0.4])))
    st = torch.cuda.Stream()
    lib.mppi_batch_graph(b, st)
    st.synchronize()
    compare(2, oracle=True)
    lib.mppi_set_terrain_weights(ctrls[0], [0.5, 0.3, 0.2])
    scs[0] = scs[0].replace(terrain_w=tuple(float(x) for x in np.float32([0.5, 0.3, 0.2])))
    lib.mppi_batch_graph(b, st)
    st.synchronize()
    compare(3)
