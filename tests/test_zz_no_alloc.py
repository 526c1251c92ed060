"""mppi_update_noalloc: the allocation-free weights-and-update entry point.

Callers that cannot allocate device memory once running (a real-time
control loop with memory fixed at start-up, or a framework that forbids its
plug-ins to call cudaMalloc) use this call instead of relying on a
controller's scratch buffers.  The test feeds it the costs from mppi_step
and the clamped sampled controls of the same iteration (the library's own
noise, clamped into the control box), and checks that its weights and U_new
agree with mppi_step's, on two calls in a row (the second call reuses the
static scratch the first one left behind).
"""
import numpy as np
import pytest

import scenarios as S
from parity import TOL_U, TOL_W, make_ctrl

pytestmark = pytest.mark.gpu


def _sampled_controls(lib, sc, U, it):
    import torch
    P = sc.params
    eps = torch.empty(P.K, P.T, 2, device="cuda")
    lib.gpmppi_control_noise(P.seed, P.K, P.T, it, P.sigma, eps)
    lo = torch.tensor(P.u_min, dtype=torch.float32, device="cuda")
    hi = torch.tensor(P.u_max, dtype=torch.float32, device="cuda")
    ut = torch.maximum(torch.minimum(U[None, :, :] + eps, hi), lo)     # (K, T, 2)
    return ut.transpose(0, 1).contiguous()                             # (T, K, 2)


def test_noalloc_update_matches_mppi_step(lib):
    import torch
    sc = S.scenario("cfg1")
    P = sc.params
    g, ctrl = make_ctrl(lib, sc)
    U = torch.tensor(sc.U0, dtype=torch.float32, device="cuda")
    for call in range(2):
        it = 10 + call
        lib.mppi_set_iteration(ctrl, it)
        U_new = torch.empty_like(U)
        w = torch.empty(P.K, device="cuda")
        c = torch.empty(P.K, device="cuda")
        lib.mppi_step(ctrl, sc.x0, U, U_new, w, c)
        ut = _sampled_controls(lib, sc, U, it)
        U_new2 = torch.full_like(U, float("nan"))
        w2 = torch.full_like(w, float("nan"))
        lib.mppi_update_noalloc(c, ut, U, U_new2, w2, P.K, P.T, P.lam)
        torch.cuda.synchronize()
        assert np.max(np.abs(U_new2.cpu().numpy() - U_new.cpu().numpy())) <= TOL_U
        assert np.max(np.abs(w2.cpu().numpy() - w.cpu().numpy())) <= TOL_W
        assert abs(float(w2.sum()) - 1.0) <= 1e-5
        U = U_new.clone()


def test_noalloc_rejects_sizes_beyond_the_array(lib):
    import torch
    x = torch.zeros(16, device="cuda")
    f = lib.load().mppi_update_noalloc
    p = lib._dptr(x)
    # ceil(K/256) * T above 65536: refused before any GPU work
    for K, T in ((256 * 65537, 1), (256 * 1024, 65)):
        rc = f(p, p, p, lib._dptr(torch.zeros(16, device="cuda")), None, K, T, 1.0, lib._stream(None))
        assert rc == lib.GPMPPI_ERR_INVALID_ARG
        assert "65536" in lib.gpmppi_last_error()


def _fp64_update(c, ut, U, lam):
    """Softmax weights and weighted update in FP64 (torch, on the host)."""
    import torch
    c64 = c.double().cpu()
    w = torch.exp(-(c64 - c64.min()) / lam)
    w = w / w.sum()
    ut64 = ut.double().cpu()                      # (T, K, 2)
    U64 = U.double().cpu()
    return U64 + torch.einsum("s,ksc->kc", w, ut64 - U64[:, None, :]), w


@pytest.mark.parametrize("K,T,with_w", [(16640, 20, True),     # 65 sample blocks: one CTA per block
                                         (65536, 256, True),    # ceil(K/256) * T = 65536, the limit
                                         (4099, 33, False)])    # ragged K, no weights output
def test_noalloc_update_sizes(lib, K, T, with_w):
    """Against an FP64 softmax and update of the same costs and controls, on
    two calls in a row: the step-blocked and the per-block grids, the size at
    the array's limit (the last partial sum next to the ticket word) and a
    NULL weights output."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(K + T)
    lam = 0.7
    for call in range(2):
        c = 50.0 + 5.0 * torch.rand(K, device="cuda", generator=g)
        ut = torch.rand(T, K, 2, device="cuda", generator=g) * 2.0 - 0.5
        U = torch.rand(T, 2, device="cuda", generator=g)
        U_new = torch.full_like(U, float("nan"))
        w = torch.full((K,), float("nan"), device="cuda") if with_w else None
        lib.mppi_update_noalloc(c, ut, U, U_new, w, K, T, lam)
        torch.cuda.synchronize()
        U_ref, w_ref = _fp64_update(c, ut, U, lam)
        assert torch.max(torch.abs(U_new.cpu().double() - U_ref)).item() <= TOL_U, f"call {call}"
        if with_w:
            assert torch.max(torch.abs(w.cpu().double() - w_ref)).item() <= TOL_W, f"call {call}"


def test_noalloc_refuses_host_and_foreign_pointers(lib):
    """Host memory where device memory is required is refused on the host
    side (GPMPPI_ERR_INVALID_ARG), before any launch."""
    import ctypes

    import torch
    K, T = 256, 4
    dev = torch.zeros(2 * K * T, device="cuda")
    host = torch.zeros(2 * K * T).pin_memory()
    plain = np.zeros(2 * K * T, dtype=np.float32)
    f = lib.load().mppi_update_noalloc
    d = lib._dptr(dev)
    d2 = lib._dptr(torch.zeros(2 * T, device="cuda"))
    for bad in (ctypes.c_void_p(host.data_ptr()), plain.ctypes.data_as(ctypes.c_void_p)):
        for args in ((bad, d, d, d2), (d, bad, d, d2), (d, d, bad, d2), (d, d, d2, bad)):
            rc = f(*args, None, K, T, 1.0, lib._stream(None))
            assert rc == lib.GPMPPI_ERR_INVALID_ARG, lib.gpmppi_last_error()
    torch.cuda.synchronize()
