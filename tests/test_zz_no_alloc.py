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
