"""GPU parity of the rollout and the MPPI step against the FP64 oracle on
small and ragged cases, plus the edge cases of the method."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from parity import (check_step, check_trace, gpu_step, gpu_trace, make_ctrl, to_np)

pytestmark = pytest.mark.gpu


def _oracle(sc, state=None, U=None, it=0, samples=None, nominal_sxy=None):
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    state = sc.x0 if state is None else state
    U = sc.U0 if U is None else U
    return O.rollout(sc, fits, state, U, it, samples=samples, nominal_sxy=nominal_sxy)


def test_trace_small_ragged(lib):
    # K = 77 over several CTAs with a ragged tail, N = 45 (not a multiple of 16)
    sc = S.scenario("small")
    g, ctrl = make_ctrl(lib, sc)
    tr = gpu_trace(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    ro = _oracle(sc)
    info = check_trace(sc, ro, tr)
    assert info["n_ambiguous_stages"] < 5
    # the trace instantiation computes the same costs as the hot path
    _, _, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    np.testing.assert_allclose(tr["costs"], c, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("name", ["small", "cfg1"])
def test_step_parity(lib, name):
    sc = S.scenario(name)
    g, ctrl = make_ctrl(lib, sc)
    U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    ro = _oracle(sc)
    info = check_step(sc, ro, sc.U0, U_new, w, c)
    assert abs(w.sum() - 1.0) < 1e-5
    assert lib.mppi_get_iteration(ctrl) == 1
    print(name, info)


def test_iteration_counter_advances_draws(lib):
    sc = S.scenario("small")
    g, ctrl = make_ctrl(lib, sc)
    lib.mppi_set_iteration(ctrl, (1 << 32) + 7)
    U1, w1, c1 = gpu_step(lib, ctrl, sc, sc.x0, sc.U0)
    U2, w2, c2 = gpu_step(lib, ctrl, sc, sc.x0, sc.U0)
    assert lib.mppi_get_iteration(ctrl) == (1 << 32) + 9
    check_step(sc, _oracle(sc, it=(1 << 32) + 7), sc.U0, U1, w1, c1)
    check_step(sc, _oracle(sc, it=(1 << 32) + 8), sc.U0, U2, w2, c2)


def test_repeat_is_deterministic(lib):
    sc = S.scenario("cfg1")
    g, ctrl = make_ctrl(lib, sc)
    a = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=4)
    b = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("case", ["K1", "T1", "N0", "O0", "P1", "clamp", "K_odd", "state"])
def test_edge_cases(lib, case):
    kw = {}
    if case == "K1":
        kw = dict(K=1)
    elif case == "T1":
        kw = dict(T=1)
    elif case == "N0":
        kw = dict(N=0)
    elif case == "O0":
        kw = dict(O=0)
    elif case == "K_odd":
        kw = dict(K=1001, T=3)
    sc = S.scenario("small", **kw)
    if case == "P1":
        sc = sc.replace(path=np.array([[1.0, 0.5]]))
    if case == "clamp":
        sc.params.sigma = (4.0, 4.0)
    state = sc.x0.copy()
    if case == "state":
        state = np.array([2.0, -1.0, 2.5, 1.9, -1.2])
    U = sc.U0.copy()
    U[:, 1] = np.linspace(-0.5, 0.5, sc.params.T)
    g, ctrl = make_ctrl(lib, sc)
    U_new, w, c = gpu_step(lib, ctrl, sc, state, U, it=2)
    ro = _oracle(sc, state=state, U=U, it=2)
    check_step(sc, ro, U, U_new, w, c)
    tr = gpu_trace(lib, ctrl, sc, state, U, it=2)
    check_trace(sc, ro, tr)
    P = sc.params
    assert np.all(U_new[:, 0] >= P.u_min[0] - 1e-6) and np.all(U_new[:, 0] <= P.u_max[0] + 1e-6)
    if case == "K1":
        assert w[0] == pytest.approx(1.0)
        np.testing.assert_allclose(U_new, ro["u_tilde"][0], atol=1e-5)


def test_nominal_mode_sequence(lib):
    # Alg. 1 Step 2: the second call tightens with Sigma propagated along the
    # first call's update
    sc = S.scenario("small", variance_mode=1)
    sc.params.sigma = (0.3, 0.3)
    g, ctrl = make_ctrl(lib, sc)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    octl = O.Controller(sc, fits)
    import torch
    U = sc.U0.copy()
    for _ in range(2):
        nom = octl.nominal_sxy.copy()
        U_new, w, c = gpu_step(lib, ctrl, sc, sc.x0, U)
        U_ref, w_ref, c_ref, ro = octl.step(sc.x0, U)
        check_step(sc, ro, U, U_new, w, c)
        sxy = torch.empty(sc.params.T, 3, device="cuda")
        lib.mppi_nominal_sxy(ctrl, sxy)
        torch.cuda.synchronize()
        ref = octl.nominal_sxy                         # along the oracle's U_new
        got = to_np(sxy)
        sf2 = sc.hyper[0].signal_var
        np.testing.assert_allclose(got[:, 0], ref[:, 0, 0], rtol=1e-3, atol=1e-6 * sf2)
        np.testing.assert_allclose(got[:, 1], ref[:, 0, 1], rtol=1e-3, atol=1e-6 * sf2)
        np.testing.assert_allclose(got[:, 2], ref[:, 1, 1], rtol=1e-3, atol=1e-6 * sf2)
        assert nom is not None
        U = U_new.astype(np.float64)


def test_error_paths_do_not_touch_the_gpu(lib):
    import torch
    sc = S.scenario("small")
    g, ctrl = make_ctrl(lib, sc)
    U = torch.tensor(sc.U0, dtype=torch.float32, device="cuda")
    U_new = torch.empty_like(U)
    # a host pointer where device memory is required
    host = np.zeros((sc.params.T, 2), dtype=np.float32)
    import ctypes
    rc = lib.load().mppi_step(ctrl.handle, sc.x0.astype(np.float32).ctypes.data_as(ctypes.c_void_p),
                              host.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(U_new.data_ptr()),
                              None, None, None)
    assert rc == lib.GPMPPI_ERR_INVALID_ARG
    # aliasing output and input
    with pytest.raises(lib.GpmppiError):
        lib.mppi_step(ctrl, sc.x0, U, U)
    # non-finite state
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_step(ctrl, np.array([0, 0, np.nan, 1, 0]), U, U_new)
    assert ei.value.code == lib.GPMPPI_ERR_NONFINITE
    # unsupported configurations
    P = S.scenario("small").params
    P.alpha = (1.0, 1.0, 0.5, 1.0, 0.5)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_create(P, sc.obstacles, sc.path, g)
    assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED
    # the controller still works afterwards
    U2, w2, c2 = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    check_step(sc, _oracle(sc), sc.U0, U2, w2, c2)


def test_closed_loop_teacher_forced(lib):
    """Receding-horizon loop of Alg. 1 run by the oracle (plant = nominal
    model + the synthetic residual); at every control step the GPU gets the
    oracle's state, nominal controls and iteration and must reproduce its
    update."""
    sc = S.scenario("cfg1", K=256, T=20)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    octl = O.Controller(sc, fits)
    g, ctrl = make_ctrl(lib, sc)
    x, U = sc.x0.copy(), sc.U0.copy()
    n_alt = 0
    for t in range(25):
        U_ref, w_ref, c_ref, ro = octl.step(x, U)
        U_new, w, c = gpu_step(lib, ctrl, sc, x, U, it=t)
        info = check_step(sc, ro, U, U_new, w, c)
        n_alt += info["n_alt"]
        x = O.mppi.plant_step(sc, x, U_ref[0], S.true_residual)
        U = O.mppi.shift_controls(U_ref)
    assert n_alt <= 5


def test_wait_expiry_reports_timeout_and_context_survives(lib):
    """Failure detection without a GPU fault: one warp of every CTA of the
    FP32 rollout waits, with a 1 ms limit, on an mbarrier that nothing arrives
    on; the wait runs out, the kernel records the timeout, that warp issues no
    copies and the kernel finishes.  The host reads GPMPPI_ERR_TIMEOUT from
    mppi_device_status (which clears it), and with the hook off and the default
    limit back the same controller steps normally, with parity against the
    oracle."""
    import torch
    sc = S.scenario("small", precision=0, K=64, N=100, T=3)
    g, ctrl = make_ctrl(lib, sc)
    assert lib.mppi_rollout_kind(ctrl) == lib.GPMPPI_KERNEL_FP32
    dev = torch.device("cuda")
    U = torch.tensor(sc.U0, dtype=torch.float32, device=dev)
    U_new = torch.empty_like(U)
    lib.mppi_set_wait_limit(ctrl, 1_000_000, expire_first=True)
    lib.mppi_set_iteration(ctrl, 0)
    lib.mppi_step(ctrl, sc.x0, U, U_new)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_device_status(ctrl)
    assert ei.value.code == lib.GPMPPI_ERR_TIMEOUT
    lib.mppi_device_status(ctrl)                 # the status word was cleared
    lib.mppi_set_wait_limit(ctrl, 2_000_000_000, expire_first=False)
    U2, w2, c2 = gpu_step(lib, ctrl, sc, sc.x0, sc.U0, it=0)
    check_step(sc, _oracle(sc), sc.U0, U2, w2, c2)
