"""GPU parity of the tensor-core (tcgen05) variance path.

First the building blocks in isolation (one CTA computes A B^T with the
library's operand layout, descriptors and TMEM path; exact 16-bit inputs, so
the FP32 result is known to rounding), then the rollout with the split
16-bit contraction against the FP64 oracle, in both 16-bit formats."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from parity import (TOL_COST, TOL_U, assert_close, check_step, check_trace, gpu_step, gpu_trace,
                    make_ctrl, reconcile_costs, trace_errors)

pytestmark = pytest.mark.gpu


def _operands(fmt, rows, K, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(rows, K, generator=g) * 2.0
    t = x.to(torch.float16 if fmt == 0 else torch.bfloat16)
    return t, t.float().double()


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("N,K", [(64, 16), (128, 32), (256, 64), (64, 48)])
@pytest.mark.parametrize("variant", [0, 2])
def test_mma_selftest(lib, fmt, N, K, variant):
    """D = A B^T on the tensor cores, A from shared memory (variant 0) or from
    tensor memory (variant 2, the cluster rollout's kernel-row operand)."""
    import torch
    A16, A = _operands(fmt, 128, K, 1)
    B16, B = _operands(fmt, N, K, 2)
    D = torch.empty(128, N, device="cuda")
    lib.gpmppi_mma_selftest(fmt, A16.cuda().view(torch.int16), B16.cuda().view(torch.int16), D,
                            variant=variant)
    ref = (A @ B.T).numpy()
    got = D.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * (1 + np.max(np.abs(ref)))


def _sc(name, precision, **kw):
    return S.scenario(name, precision=precision, **kw)


@pytest.mark.parametrize("precision", [2, 1, 3])
@pytest.mark.parametrize("name,kw", [("small", {}), ("cfg1", {}), ("small", dict(N=0)),
                                     ("small", dict(K=130, N=200)), ("small", dict(K=1, T=2))])
def test_mma_rollout_parity(lib, precision, name, kw):
    sc = _sc(name, precision, **kw)
    g, ctrl = make_ctrl(lib, sc)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = sc.U0.copy()
    U[:, 1] = 0.3 * np.cos(np.arange(sc.params.T))
    ro = O.rollout(sc, fits, sc.x0, U, 2)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=2)
    info_t = check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=2)
    info_s = check_step(sc, ro, U, U_new, w, c)
    np.testing.assert_allclose(tr["costs"], c, rtol=1e-6, atol=1e-6)
    print(name, kw, "precision", precision, info_t, info_s)


@pytest.mark.parametrize("N", [500, 2048])
def test_variance_error_per_precision(lib, N):
    """Per-quantity error against the FP64 oracle for each arithmetic of the
    variance contraction: the GP variance s(0) (the v-v entry of Sigma after
    the first step is exactly s(0)), means, covariances, margins, costs."""
    errs = {}
    for precision in (0, 2, 1, 3):
        sc = _sc("cfg2", precision, K=384, N=N, T=20)
        g, ctrl = make_ctrl(lib, sc)
        fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
        ro = O.rollout(sc, fits, sc.x0, sc.U0, 0)
        tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=0)
        sf2 = sc.hyper[0].signal_var
        var_err = float(np.max(np.abs(tr["sigma"][:, 0, 12] - ro["var"][:, 0, 0])) / sf2)
        # FP32 and the FP16 split meet the full parity tolerances; the BF16
        # split is the coarse mode and is only reported
        info = check_trace(sc, ro, tr) if precision != 1 else trace_errors(sc, ro, tr)
        ref_c, _ = reconcile_costs(sc, ro, tr["costs"])
        info["err_cost"] = float(np.max(np.abs(tr["costs"] - ref_c) / (np.abs(ref_c) + 1)))
        info["err_var_over_sf2"] = var_err
        errs[precision] = info
        print(f"N={N} precision {precision}: {info}")
    # FP32, the FP16 split and the three-term BF16 split stay inside the
    # declared GP-variance tolerance (1e-4 sf2) and pass every parity check
    # above; the two-term BF16 split is reported
    assert errs[0]["err_var_over_sf2"] <= 1e-4
    assert errs[2]["err_var_over_sf2"] <= 1e-4
    assert errs[3]["err_var_over_sf2"] <= 1e-4
    assert errs[1]["err_var_over_sf2"] <= 1e-3


@pytest.mark.parametrize("precision", [2])
def test_mma_cfg3_sampled_and_properties(lib, precision):
    sc = _sc("cfg3", precision)
    P = sc.params
    g, ctrl = make_ctrl(lib, sc)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([[0, 127, 128, P.K - 1], rng.integers(0, P.K, 16)]))
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 1, samples=rows)
    check_trace(sc, ro, tr, rows)
    ref_c, _ = reconcile_costs(sc, ro, tr["costs"][rows], rows)
    assert_close(tr["costs"][rows], ref_c, TOL_COST, what="costs")
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    np.testing.assert_allclose(c, tr["costs"], rtol=1e-6, atol=1e-6)
    assert np.max(np.abs(w - O.mppi_weights(c, P.lam))) <= 1e-5
    ut = np.empty((P.K, P.T, 2))
    for k in range(P.T):
        eps = O.control_noise(P.seed, k, np.arange(P.K), 1, P.sigma)
        ut[:, k] = np.clip(sc.U0[k] + eps, P.u_min, P.u_max)
    U_chk = sc.U0 + np.einsum("s,skc->kc", w, ut - sc.U0[None])
    assert np.max(np.abs(U_new - U_chk)) <= TOL_U


@pytest.mark.parametrize("rps", [2, 4, 8])
def test_mma_threads_per_sample_layouts(lib, rps, monkeypatch):
    """Every producer layout (128, 64 or 32 samples per CTA) gives the same
    parity; K = 300 spans several CTAs with a ragged tail in each layout."""
    monkeypatch.setenv("GPMPPI_MMA_THREADS_PER_SAMPLE", str(rps))
    monkeypatch.setenv("GPMPPI_NO_CLUSTER", "1")      # the streaming kernel's layouts
    sc = _sc("small", 2, K=300, N=333, T=6)
    g, ctrl = make_ctrl(lib, sc)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 5)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=5)
    check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=5)
    check_step(sc, ro, sc.U0, U_new, w, c)


def test_mma_scene_too_large_for_shared_memory(lib):
    """A scene whose segments and obstacles do not fit next to the pipeline
    is read from global memory: same parity."""
    sc = _sc("small", 2, K=70, N=1900, T=3, O=1500)
    t = np.linspace(0, 2 * np.pi, 6000)
    sc = sc.replace(path=np.stack([6 * np.cos(t), 3 * np.sin(t)], axis=1))
    g, ctrl = make_ctrl(lib, sc)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 1)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    check_trace(sc, ro, tr)


def test_rollout_kind_per_workload(lib):
    """Split precisions with N <= 512 take the cluster kernel (its factor share
    resident in shared memory), larger N the streaming kernel, FP32 the CUDA
    cores and terrain ensembles their own rollout."""
    cases = [(_sc("small", 2, N=500), lib.GPMPPI_KERNEL_TC_CLUSTER),
             (_sc("small", 1, N=100), lib.GPMPPI_KERNEL_TC_CLUSTER),
             (_sc("small", 2, N=700), lib.GPMPPI_KERNEL_TC_STREAM),
             (_sc("small", 0), lib.GPMPPI_KERNEL_FP32),
             (S.terrain_scenario("small", M=2, N=30), lib.GPMPPI_KERNEL_ENSEMBLE)]
    for sc, kind in cases:
        _, ctrl = make_ctrl(lib, sc)
        assert lib.mppi_rollout_kind(ctrl) == kind


@pytest.mark.parametrize("N", [100, 200, 333, 512])
@pytest.mark.parametrize("precision", [2, 1])
def test_cluster_kernel_parity_and_streaming_agreement(lib, N, precision, monkeypatch):
    """Cluster sizes 1, 2, 4 (N <= 128, <= 256, <= 512) against the oracle, and
    the same controller on the streaming kernel: same costs and update."""
    sc = _sc("small", precision, K=300, N=N, T=6)
    g, ctrl = make_ctrl(lib, sc)
    assert lib.mppi_rollout_kind(ctrl) == lib.GPMPPI_KERNEL_TC_CLUSTER
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = sc.U0.copy()
    U[:, 1] = 0.4 * np.sin(np.arange(sc.params.T))
    ro = O.rollout(sc, fits, sc.x0, U, 3)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=3)
    check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=3)
    check_step(sc, ro, U, U_new, w, c)
    monkeypatch.setenv("GPMPPI_NO_CLUSTER", "1")
    _, ctrl2 = make_ctrl(lib, sc, g)
    assert lib.mppi_rollout_kind(ctrl2) == lib.GPMPPI_KERNEL_TC_STREAM
    U2, w2, c2 = gpu_step(lib, ctrl2, sc, sc.x0, U, it=3)
    np.testing.assert_allclose(c2, c, rtol=1e-5, atol=1e-5)
    assert np.max(np.abs(U2 - U_new)) <= TOL_U


@pytest.mark.parametrize("K,T", [(1, 1), (129, 2), (130, 3), (257, 5)])
def test_cluster_kernel_edges(lib, K, T):
    """Four-CTA clusters (N = 500) at the edges of the step pipeline: one step
    (no noise computed ahead, no record handed over while another is pending),
    two and three steps (the two-slot rings wrap), one sample (127 idle rows of
    the MMA tile) and a second sample tile with one or two live samples."""
    sc = _sc("small", 2, K=K, N=500, T=T)
    g, ctrl = make_ctrl(lib, sc)
    assert lib.mppi_rollout_kind(ctrl) == lib.GPMPPI_KERNEL_TC_CLUSTER
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = sc.U0.copy()
    ro = O.rollout(sc, fits, sc.x0, U, 5)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, U, it=5)
    check_trace(sc, ro, tr)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U, it=5)
    check_step(sc, ro, U, U_new, w, c)


def test_cluster_kernel_scene_in_global_memory(lib):
    """A scene too large to stage next to the resident factor share is read
    from global memory by the cluster kernel: same parity."""
    sc = _sc("small", 2, K=150, N=400, T=3, O=1500)
    t = np.linspace(0, 2 * np.pi, 6000)
    sc = sc.replace(path=np.stack([6 * np.cos(t), 3 * np.sin(t)], axis=1))
    g, ctrl = make_ctrl(lib, sc)
    assert lib.mppi_rollout_kind(ctrl) == lib.GPMPPI_KERNEL_TC_CLUSTER
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    ro = O.rollout(sc, fits, sc.x0, sc.U0, 1)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=1)
    check_trace(sc, ro, tr)


@pytest.mark.parametrize("K", [16384, 16700, 65800])
def test_update_sample_block_counts(lib, K):
    """The update over 64, 66 (last block ragged) and 258 sample blocks (more
    blocks than the combining CTA has threads), each with two step blocks of
    16 steps: weights against Alg. 1's softmax of the returned costs, U_new
    against the weighted sum over the oracle's perturbed controls."""
    sc = _sc("small", 2, K=K, N=100, T=20)
    P = sc.params
    g, ctrl = make_ctrl(lib, sc)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=3)
    assert np.all(np.isfinite(c))
    assert np.max(np.abs(w - O.mppi_weights(c, P.lam))) <= 1e-5
    ut = np.empty((P.K, P.T, 2))
    for k in range(P.T):
        eps = O.control_noise(P.seed, k, np.arange(P.K), 3, P.sigma)
        ut[:, k] = np.clip(sc.U0[k] + eps, P.u_min, P.u_max)
    U_chk = sc.U0 + np.einsum("s,skc->kc", w, ut - sc.U0[None])
    assert np.max(np.abs(U_new - U_chk)) <= TOL_U
