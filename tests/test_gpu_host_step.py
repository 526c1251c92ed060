"""mppi_step_host: one MPPI iteration (Alg. 1 Step 1) with every array on the host.

A receding-horizon controller holds U on the host between control periods.
The host-buffer call must give bit-identical results to mppi_step on device
buffers at the same iteration, for every rollout kernel (FP32, cluster,
streaming), with numpy arrays and with pinned tensors. It must also refuse
device pointers.
"""
import numpy as np
import pytest

import scenarios as S
from parity import make_ctrl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,no_cluster", [(0, False), (2, False), (2, True)])
def test_host_step_equals_device_step(lib, precision, no_cluster, monkeypatch):
    import torch
    if no_cluster:
        monkeypatch.setenv("GPMPPI_NO_CLUSTER", "1")
    sc = S.scenario("small", precision=precision, K=300, N=333, T=12)
    P = sc.params
    g, ctrl = make_ctrl(lib, sc)
    U0 = np.ascontiguousarray(sc.U0, dtype=np.float32)
    for it in (3, 4):
        lib.mppi_set_iteration(ctrl, it)
        U = torch.tensor(U0, device="cuda")
        U_new = torch.empty_like(U)
        w = torch.empty(P.K, device="cuda")
        c = torch.empty(P.K, device="cuda")
        lib.mppi_step(ctrl, sc.x0, U, U_new, w, c)
        torch.cuda.synchronize()

        lib.mppi_set_iteration(ctrl, it)
        U_new_h = np.full_like(U0, np.nan)
        w_h = np.full(P.K, np.nan, dtype=np.float32)
        c_h = np.full(P.K, np.nan, dtype=np.float32)
        lib.mppi_step_host(ctrl, sc.x0, U0, U_new_h, w_h, c_h)
        assert np.array_equal(U_new_h, U_new.cpu().numpy())
        assert np.array_equal(w_h, w.cpu().numpy())
        assert np.array_equal(c_h, c.cpu().numpy())
        assert lib.mppi_get_iteration(ctrl) == it + 1

        # pinned tensors, no weights or costs
        lib.mppi_set_iteration(ctrl, it)
        U_p = torch.tensor(U0).pin_memory()
        out_p = torch.full_like(U_p, float("nan")).pin_memory()
        lib.mppi_step_host(ctrl, sc.x0, U_p, out_p)
        assert np.array_equal(out_p.numpy(), U_new.cpu().numpy())


def test_host_step_refuses_device_buffers(lib):
    import torch
    sc = S.scenario("small", precision=0, K=64, N=50, T=5)
    g, ctrl = make_ctrl(lib, sc)
    U = np.ascontiguousarray(sc.U0, dtype=np.float32)
    out = np.empty_like(U)
    with pytest.raises(ValueError):
        lib.mppi_step_host(ctrl, sc.x0, torch.tensor(U, device="cuda"), out)
    # through the C ABI directly: a device pointer is INVALID_ARG, nothing runs
    d = torch.tensor(U, device="cuda")
    st = np.ascontiguousarray(sc.x0, dtype=np.float32)
    rc = lib.load().mppi_step_host(ctrl.handle, st.ctypes.data, lib._dptr(d), out.ctypes.data,
                                   None, None, None)
    assert rc == lib.GPMPPI_ERR_INVALID_ARG
    assert lib.mppi_get_iteration(ctrl) == 0
