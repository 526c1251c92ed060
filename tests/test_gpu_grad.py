"""Adjoint rollout (gradient of the sigmoid-smoothed chance-constrained cost)
against the FP64 oracle: central differences at h = 1e-3 and the oracle's
FP64 gradient (h = 1e-6), in the nominal controls U and the GP lengthscales,
plus the GPU's own directional differences and the autograd wrapper."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gradcases import tiny
from parity import make_ctrl, to_np

pytestmark = pytest.mark.gpu

SLOPE = 20.0
TOL_GRAD = 1e-3        # relative, per component, floored at 0.1% of the largest component
TOL_J = 1e-4


def grad_err(g, ref):
    """Largest |g - ref| / max(|ref|, 1e-3 max |ref|): every component of at
    least 0.1% of the largest is held to the relative tolerance; smaller ones
    to an absolute error of TOL_GRAD * 1e-3 * max |ref| (their FP32 sums are
    rounded at the scale of the largest terms)."""
    g, ref = np.asarray(g, dtype=np.float64).ravel(), np.asarray(ref, dtype=np.float64).ravel()
    floor = 1e-3 * np.max(np.abs(ref))
    return float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor)))


def grad_err_unfloored(g, ref):
    """Per-component relative errors |g - ref| / |ref| (reported, not asserted)."""
    g, ref = np.asarray(g, dtype=np.float64).ravel(), np.asarray(ref, dtype=np.float64).ravel()
    return np.abs(g - ref) / np.maximum(np.abs(ref), 1e-30)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def gpu_grad(lib, ctrl, sc, U, weights=None, want_dl=True):
    import torch
    Ud = torch.tensor(np.asarray(U), dtype=torch.float32, device="cuda")
    w = None if weights is None else torch.tensor(weights, dtype=torch.float32, device="cuda")
    J, dU, dl = lib.mppi_grad(ctrl, sc.x0, Ud, SLOPE, w, want_dl=want_dl)
    torch.cuda.synchronize()
    return float(to_np(J)[0]), to_np(dU), (to_np(dl) if dl is not None else None)


def _shared(sc):
    h = sc.hyper[0]
    return sc.replace(hyper=(h, S.Hyper(tuple(h.lengthscale), h.signal_var, h.noise_var)))


def test_grad_tiny_matches_oracle(lib):
    sc = tiny(shared=True)
    _, ctrl = make_ctrl(lib, sc)
    J, dU, dl = gpu_grad(lib, ctrl, sc, sc.U0)
    x0, U = f32(sc.x0), f32(sc.U0)
    Jo, _ = O.objective(sc, sc.hyper, x0, U, 0, None, SLOPE)
    gU, gL = O.fd_gradient(sc, sc.hyper, x0, U, 0, None, SLOPE)
    assert abs(J - Jo) <= TOL_J * abs(Jo)
    eU, eL = grad_err(dU, gU), grad_err(dl, gL)
    print("tiny", J, Jo, eU, eL)
    assert eU <= TOL_GRAD and eL <= TOL_GRAD


def test_grad_small_all_samples(lib):
    """K=77 (ragged last CTA), T=7 (segments of 3, 3, 1), N=45, six obstacles."""
    sc = _shared(S.scenario("small"))
    U = sc.U0.copy()
    U[:, 1] = 0.5 * np.sin(np.arange(sc.params.T))
    _, ctrl = make_ctrl(lib, sc)
    J, dU, dl = gpu_grad(lib, ctrl, sc, U)
    x0, U64 = f32(sc.x0), f32(U)
    Jo, _ = O.objective(sc, sc.hyper, x0, U64, 0, None, SLOPE)
    gU, gL = O.fd_gradient(sc, sc.hyper, x0, U64, 0, None, SLOPE)
    hU, hL = O.fd_gradient(sc, sc.hyper, x0, U64, 0, None, SLOPE, h_u=1e-3, h_l=1e-3)
    print("small", J, Jo, grad_err(dU, gU), grad_err(dl, gL), grad_err(dU, hU), grad_err(dl, hL))
    assert abs(J - Jo) <= TOL_J * abs(Jo)
    assert grad_err(dU, gU) <= TOL_GRAD
    assert grad_err(dl, gL) <= TOL_GRAD
    assert grad_err(dU, hU) <= TOL_GRAD
    assert grad_err(dl, hL) <= TOL_GRAD


def test_grad_weights_select_samples(lib):
    """The weighted objective sum_s w_s S_s over a subset equals the oracle's mean over it."""
    sc = _shared(S.scenario("small", K=200, T=5, N=60, O=4, seed=9))
    _, ctrl = make_ctrl(lib, sc)
    sub = np.array([3, 17, 64, 128, 199])
    w = np.zeros(sc.params.K)
    w[sub] = 1.0 / len(sub)
    J, dU, dl = gpu_grad(lib, ctrl, sc, sc.U0, weights=w)
    x0, U64 = f32(sc.x0), f32(sc.U0)
    Jo, _ = O.objective(sc, sc.hyper, x0, U64, 0, sub, SLOPE)
    gU, gL = O.fd_gradient(sc, sc.hyper, x0, U64, 0, sub, SLOPE)
    assert abs(J - Jo) <= TOL_J * abs(Jo)
    assert grad_err(dU, gU) <= TOL_GRAD
    assert grad_err(dl, gL) <= TOL_GRAD


def test_grad_cfg4_sampled(lib):
    """The differentiable workload (K=4096, T=50, N=1000, 16 obstacles, slope 20)
    with the objective restricted to eight samples by the weights, so that the
    oracle can difference it: all lengthscale components and 16 control
    components, at h = 1e-3 and against the FP64 gradient (h = 1e-6)."""
    sc = _shared(S.scenario("cfg4"))
    P = sc.params
    U = sc.U0.copy()
    U[:, 1] = 0.4 * np.sin(np.arange(P.T) / 6.0)
    _, ctrl = make_ctrl(lib, sc)
    rng = np.random.default_rng(4)
    sub = np.sort(rng.choice(P.K, 8, replace=False))
    w = np.zeros(P.K)
    w[sub] = 1.0 / len(sub)
    J, dU, dl = gpu_grad(lib, ctrl, sc, U, weights=w)
    x0, U64 = f32(sc.x0), f32(U)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    Jo, _ = O.objective(sc, sc.hyper, x0, U64, 0, sub, SLOPE, fits)
    assert abs(J - Jo) <= TOL_J * abs(Jo)
    comps = rng.choice(2 * P.T, 16, replace=False)
    ref = {1e-3: [], 1e-6: []}
    for h in ref:
        for cidx in comps:
            k, c = divmod(int(cidx), 2)
            Up, Um = U64.copy(), U64.copy()
            Up[k, c] += h
            Um[k, c] -= h
            jp, _ = O.objective(sc, sc.hyper, x0, Up, 0, sub, SLOPE, fits)
            jm, _ = O.objective(sc, sc.hyper, x0, Um, 0, sub, SLOPE, fits)
            ref[h].append((jp - jm) / (2 * h))
    gpu_u = dU.reshape(-1)[comps]
    # floor for the sampled components: 0.1% of the largest |dJ/dU| on the GPU
    floor = 1e-3 * np.max(np.abs(dU))
    for h, vals in ref.items():
        vals = np.array(vals)
        err = np.max(np.abs(gpu_u - vals) / np.maximum(np.abs(vals), floor))
        print("cfg4 dU", h, err, "unfloored max", float(np.max(grad_err_unfloored(gpu_u, vals))),
              "min |ref| / max |ref|", float(np.min(np.abs(vals)) / np.max(np.abs(vals))))
        assert err <= TOL_GRAD
    for h in (1e-3, 1e-6):
        gL = np.zeros((2, 4))
        for o in range(2):
            for d in range(4):
                jp, _ = O.objective(sc, O.with_lengthscale(sc.hyper, o, d, h), x0, U64, 0, sub, SLOPE)
                jm, _ = O.objective(sc, O.with_lengthscale(sc.hyper, o, d, -h), x0, U64, 0, sub, SLOPE)
                gL[o, d] = (jp - jm) / (2 * h)
        print("cfg4 dl", h, grad_err(dl, gL), "unfloored", grad_err_unfloored(dl, gL).tolist(),
              dl.ravel(), gL.ravel())
        assert grad_err(dl, gL) <= TOL_GRAD


def test_grad_directional_difference_on_gpu(lib):
    """All 4096 samples of the differentiable workload: the adjoint's dJ/dU
    along a random direction against central differences of the GPU's own
    objective (h = 1e-3)."""
    import torch
    sc = _shared(S.scenario("cfg4"))
    P = sc.params
    U = sc.U0.copy()
    U[:, 1] = 0.4 * np.sin(np.arange(P.T) / 6.0)
    _, ctrl = make_ctrl(lib, sc)
    J, dU, dl = gpu_grad(lib, ctrl, sc, U, want_dl=False)
    rng = np.random.default_rng(7)
    d = rng.standard_normal(U.shape)
    d /= np.linalg.norm(d)
    h = 1e-3
    vals = []
    for sgn in (1.0, -1.0):
        Ud = torch.tensor(U + sgn * h * d, dtype=torch.float32, device="cuda")
        Jt, _, _ = lib.mppi_grad(ctrl, sc.x0, Ud, SLOPE, want_dU=False)
        vals.append(float(to_np(Jt)[0]))
    fd = (vals[0] - vals[1]) / (2 * h)
    ad = float(np.sum(dU * d))
    print("directional", ad, fd)
    assert abs(ad - fd) <= 5e-3 * max(abs(fd), 0.05 * np.linalg.norm(dU))


def test_autograd_function_and_determinism(lib):
    import torch
    sc = _shared(S.scenario("small"))
    _, ctrl = make_ctrl(lib, sc)
    U = torch.tensor(sc.U0, dtype=torch.float32, device="cuda", requires_grad=True)
    ell = torch.tensor([list(h.lengthscale) for h in sc.hyper], dtype=torch.float32, device="cuda",
                       requires_grad=True)
    J = lib.smoothed_rollout_cost(ctrl, sc.x0, U, ell, slope=SLOPE)
    (3.0 * J).backward()
    J2, dU, dl = lib.mppi_grad(ctrl, sc.x0, U.detach(), SLOPE)
    torch.cuda.synchronize()
    assert float(J.detach()) == float(J2[0])
    assert torch.equal(U.grad, 3.0 * dU)
    assert torch.equal(ell.grad, 3.0 * dl)
    J3, dU3, dl3 = lib.mppi_grad(ctrl, sc.x0, U.detach(), SLOPE)
    assert torch.equal(dU3, dU) and torch.equal(dl3, dl) and torch.equal(J3, J2)
    # only U: no lengthscale work
    U.grad = None
    J4 = lib.smoothed_rollout_cost(ctrl, sc.x0, U, slope=SLOPE)
    J4.backward()
    assert torch.equal(U.grad, dU)
    with pytest.raises(ValueError):
        lib.smoothed_rollout_cost(ctrl, sc.x0, U, ell * 1.5, slope=SLOPE)


def test_grad_rejects_bad_arguments(lib):
    import torch
    sc = S.scenario("small", variance_mode=1)
    _, ctrl = make_ctrl(lib, sc)
    U = torch.tensor(sc.U0, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_grad(ctrl, sc.x0, U, SLOPE)
    assert ei.value.code == lib.GPMPPI_ERR_UNSUPPORTED
    sc = S.scenario("small")
    _, ctrl = make_ctrl(lib, sc)
    with pytest.raises(lib.GpmppiError) as ei:
        lib.mppi_grad(ctrl, sc.x0, U, -1.0)
    assert ei.value.code == lib.GPMPPI_ERR_INVALID_ARG
    J = torch.empty(1, device="cuda")
    dl = torch.empty(8, device="cuda")
    import ctypes
    st = np.asarray(sc.x0, dtype=np.float32)
    rc = lib.load().mppi_grad(ctrl.handle, st.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(U.data_ptr()),
                              None, ctypes.c_float(SLOPE), ctypes.c_void_p(J.data_ptr()), None,
                              ctypes.c_void_p(dl.data_ptr()), None)
    assert rc == lib.GPMPPI_ERR_INVALID_ARG
