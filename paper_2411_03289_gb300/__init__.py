"""Python binding of libgpmppi, the GB300 chance-constrained GP-MPPI rollout.

Argument marshalling only: every step of the rollout, the GP fit and the
MPPI update runs in the CUDA kernels behind the C ABI of include/gpmppi.h.
The functions carry the C names; device arrays are torch CUDA tensors (their
data pointers are passed through), host arrays are numpy arrays, and
``stream`` defaults to torch's current CUDA stream.  There is no CPU path: if
the shared library has not been built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB_PATH

GPMPPI_OK = 0
GPMPPI_ERR_INVALID_ARG = -1
GPMPPI_ERR_NOT_PD = -2
GPMPPI_ERR_CUDA = -3
GPMPPI_ERR_OOM = -4
GPMPPI_ERR_TIMEOUT = -5
GPMPPI_ERR_NONFINITE = -6
GPMPPI_ERR_UNSUPPORTED = -7
GPMPPI_VAR_PER_SAMPLE = 0
GPMPPI_VAR_NOMINAL = 1
GPMPPI_FP32 = 0
GPMPPI_BF16_SPLIT = 1
GPMPPI_FP16_SPLIT = 2
GPMPPI_BF16_SPLIT3 = 3
GPMPPI_KERNEL_FP32 = 0
GPMPPI_KERNEL_TC_STREAM = 1
GPMPPI_KERNEL_TC_CLUSTER = 2
GPMPPI_KERNEL_ENSEMBLE = 3

# names every build of the library exports (checked by the CPU test suite)
EXPORTS = ("gp_fit", "gp_destroy", "gp_factors", "gp_predict", "mppi_create", "mppi_step", "mppi_step_host",
           "mppi_rollout_trace", "mppi_set_iteration", "mppi_get_iteration", "mppi_nominal_sxy",
           "mppi_destroy", "mppi_rollout_kind", "mppi_set_wait_limit", "mppi_set_profiling", "mppi_last_profile", "mppi_device_status", "mppi_grad",
           "mppi_create_ensemble", "mppi_set_terrain_weights", "terrain_weights",
           "mppi_update_noalloc", "mppi_batch_create",
           "mppi_batch_buffers", "mppi_batch_step", "mppi_batch_graph", "mppi_batch_autotune", "mppi_batch_layout",
           "mppi_batch_get_iteration", "mppi_batch_destroy", "gpmppi_philox", "gpmppi_control_noise", "gpmppi_mma_selftest", "gpmppi_alu_probe", "gpmppi_last_error",
           "gpmppi_version")


class GpmppiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Hyper(ctypes.Structure):
    _fields_ = [("lengthscale", ctypes.c_double * 4), ("signal_var", ctypes.c_double),
                ("noise_var", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("T", ctypes.c_int32), ("dt", ctypes.c_float),
                ("tau_v", ctypes.c_float), ("tau_w", ctypes.c_float),
                ("sigma", ctypes.c_float * 2), ("lambda_", ctypes.c_float),
                ("p_x", ctypes.c_float), ("u_min", ctypes.c_float * 2),
                ("u_max", ctypes.c_float * 2), ("alpha", ctypes.c_float * 5),
                ("beta", ctypes.c_float * 4), ("P_lane", ctypes.c_float),
                ("P_coll", ctypes.c_float), ("lane_half_width", ctypes.c_float),
                ("v_desired", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("variance_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("goal", ctypes.c_float * 2), ("goal_radius", ctypes.c_float),
                ("P_goal", ctypes.c_float)]


_lib = None


def load():
    """Load the shared library (it must have been built with build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgpmppi is not built ({LIB_PATH} missing): "
                           "run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
    sig = {
        "gp_fit": [vp, vp, i32, vp, ctypes.POINTER(vp)],
        "gp_destroy": [vp],
        "gp_factors": [vp, i32, vp, vp],
        "gp_predict": [vp, vp, i32, vp, vp, vp],
        "mppi_create": [vp, vp, i32, vp, i32, vp, ctypes.POINTER(vp)],
        "mppi_step": [vp, vp, vp, vp, vp, vp, vp],
        "mppi_step_host": [vp, vp, vp, vp, vp, vp, vp],
        "mppi_rollout_trace": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "mppi_set_iteration": [vp, u64],
        "mppi_get_iteration": [vp, ctypes.POINTER(u64)],
        "mppi_nominal_sxy": [vp, vp, vp],
        "mppi_destroy": [vp],
        "mppi_rollout_kind": [vp, vp],
        "mppi_set_wait_limit": [vp, u64, i32],
        "mppi_set_profiling": [vp, i32],
        "mppi_last_profile": [vp, vp, vp],
        "mppi_device_status": [vp],
        "mppi_grad": [vp, vp, vp, vp, ctypes.c_float, vp, vp, vp, vp],
        "mppi_create_ensemble": [vp, vp, i32, vp, i32, vp, i32, vp, ctypes.POINTER(vp)],
        "mppi_set_terrain_weights": [vp, vp, i32],
        "terrain_weights": [vp, vp, vp, vp, i32, i32, vp, ctypes.c_double, vp],
        "mppi_batch_create": [vp, i32, ctypes.POINTER(vp)],
        "mppi_batch_buffers": [vp, i32, vp, vp, vp, vp, vp],
        "mppi_batch_step": [vp, vp],
        "mppi_batch_graph": [vp, vp],
        "mppi_batch_autotune": [vp, vp, vp],
        "mppi_batch_layout": [vp, i32, vp, vp],
        "mppi_batch_get_iteration": [vp, i32, ctypes.POINTER(u64)],
        "mppi_batch_destroy": [vp],
        "mppi_update_noalloc": [vp, vp, vp, vp, vp, i32, i32, ctypes.c_float, vp],
        "gpmppi_philox": [u64, vp, i32, vp, vp],
        "gpmppi_control_noise": [u64, i32, i32, u64, vp, vp, vp],
        "gpmppi_mma_selftest": [i32, i32, i32, i32, vp, vp, vp],
        "gpmppi_alu_probe": [i32, i32, i32, vp, vp],
        "gpmppi_version": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.gpmppi_last_error.argtypes = []
    lib.gpmppi_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def gpmppi_last_error() -> str:
    return load().gpmppi_last_error().decode()


def gpmppi_version() -> int:
    return load().gpmppi_version()


def _check(rc):
    if rc != GPMPPI_OK:
        raise GpmppiError(rc, gpmppi_last_error())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, numel=None, name="array"):
    """Data pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    import torch
    if t.device.index is not None and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} lives on {t.device}, not on the current device "
                         f"cuda:{torch.cuda.current_device()}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def _hptr(t, numel, name, writable=False):
    """Data pointer of a contiguous float32 host array: a CPU tensor (pinned
    or not) or a numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32 or not t.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be a C-contiguous float32 array")
        if writable and not t.flags["WRITEABLE"]:
            raise ValueError(f"{name} must be writable")
        if t.size < numel:
            raise ValueError(f"{name} needs at least {numel} elements")
        return ctypes.c_void_p(t.ctypes.data)
    import torch
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must have dtype torch.float32")
    if t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host tensor")
    if t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def make_hyper(h) -> Hyper:
    out = Hyper()
    out.lengthscale[:] = [float(v) for v in h.lengthscale]
    out.signal_var = float(h.signal_var)
    out.noise_var = float(h.noise_var)
    return out


def make_params(p) -> Params:
    """Params from any object with the field names of gpmppi_params (``lam`` or
    ``lambda_`` for the temperature)."""
    out = Params()
    out.K, out.T = int(p.K), int(p.T)
    out.dt, out.tau_v, out.tau_w = float(p.dt), float(p.tau_v), float(p.tau_w)
    out.sigma[:] = [float(v) for v in p.sigma]
    out.lambda_ = float(getattr(p, "lam", getattr(p, "lambda_", 1.0)))
    out.p_x = float(p.p_x)
    out.u_min[:] = [float(v) for v in p.u_min]
    out.u_max[:] = [float(v) for v in p.u_max]
    out.alpha[:] = [float(v) for v in p.alpha]
    out.beta[:] = [float(v) for v in p.beta]
    out.P_lane, out.P_coll = float(p.P_lane), float(p.P_coll)
    out.lane_half_width, out.v_desired = float(p.lane_half_width), float(p.v_desired)
    out.seed = int(p.seed) & 0xFFFFFFFFFFFFFFFF
    out.variance_mode = int(p.variance_mode)
    out.precision = int(p.precision)
    out.goal[:] = [float(v) for v in getattr(p, "goal", (0.0, 0.0))]
    out.goal_radius = float(getattr(p, "goal_radius", 0.5))
    out.P_goal = float(getattr(p, "P_goal", 100.0))
    return out


class GP:
    """Owning wrapper of a gpmppi_gp handle."""

    def __init__(self, handle, N, hyper=None):
        self.handle, self.N, self.hyper = handle, N, hyper

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.gp_destroy(self.handle)
            self.handle = None


class Ctrl:
    """Owning wrapper of a gpmppi_ctrl handle (keeps its GP alive)."""

    def __init__(self, handle, gp, K, T):
        self.handle, self.gp, self.K, self.T = handle, gp, K, T

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mppi_destroy(self.handle)
            self.handle = None


def gp_fit(X, Y, hyper) -> GP:
    lib = load()
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 4))
    Y = np.ascontiguousarray(np.asarray(Y, dtype=np.float64).reshape(-1, 2))
    if X.shape[0] != Y.shape[0]:
        raise ValueError("X and Y row counts differ")
    hy = (Hyper * 2)(make_hyper(hyper[0]), make_hyper(hyper[1]))
    h = ctypes.c_void_p()
    _check(lib.gp_fit(X.ctypes.data_as(ctypes.c_void_p), Y.ctypes.data_as(ctypes.c_void_p),
                      X.shape[0], ctypes.cast(hy, ctypes.c_void_p), ctypes.byref(h)))
    return GP(h.value, X.shape[0], hyper)


def gp_destroy(gp: GP):
    if gp.handle:
        _check(load().gp_destroy(gp.handle))
        gp.handle = None


def gp_factors(gp: GP, j: int):
    """(Linv (N,N), alpha (N,)) in float64 copied from the device."""
    N = gp.N
    Linv = np.zeros((N, N))
    alpha = np.zeros(N)
    _check(load().gp_factors(gp.handle, j, Linv.ctypes.data_as(ctypes.c_void_p),
                             alpha.ctypes.data_as(ctypes.c_void_p)))
    return Linv, alpha


def gp_predict(gp: GP, Z, mean, var, stream=None):
    M = Z.shape[0]
    _check(load().gp_predict(gp.handle, _dptr(Z, numel=4 * M, name="Z"), M,
                             _dptr(mean, numel=2 * M, name="mean"),
                             _dptr(var, numel=2 * M, name="var"), _stream(stream)))


def mppi_create(params, obstacles, path, gp: GP) -> Ctrl:
    lib = load()
    p = make_params(params)
    obst = _f32(obstacles).reshape(-1, 3)
    pth = _f32(path).reshape(-1, 2)
    h = ctypes.c_void_p()
    _check(lib.mppi_create(ctypes.byref(p), obst.ctypes.data_as(ctypes.c_void_p) if obst.size else None,
                           obst.shape[0], pth.ctypes.data_as(ctypes.c_void_p), pth.shape[0],
                           gp.handle, ctypes.byref(h)))
    return Ctrl(h.value, gp, p.K, p.T)


def mppi_create_ensemble(params, obstacles, path, gps, weights) -> Ctrl:
    """Controller over the terrain ensemble of Eq. 3 (gps: list of GP, weights: M floats)."""
    lib = load()
    p = make_params(params)
    obst = _f32(obstacles).reshape(-1, 3)
    pth = _f32(path).reshape(-1, 2)
    M = len(gps)
    handles = (ctypes.c_void_p * M)(*[g.handle for g in gps])
    w = _f32(weights).reshape(M)
    h = ctypes.c_void_p()
    _check(lib.mppi_create_ensemble(ctypes.byref(p), obst.ctypes.data_as(ctypes.c_void_p) if obst.size else None,
                                    obst.shape[0], pth.ctypes.data_as(ctypes.c_void_p), pth.shape[0],
                                    ctypes.cast(handles, ctypes.c_void_p), M,
                                    w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
    c = Ctrl(h.value, gps[0], p.K, p.T)
    c.terrain_gps = list(gps)       # keep every terrain GP alive with the controller
    return c


def mppi_set_terrain_weights(ctrl: Ctrl, weights):
    w = _f32(weights).reshape(-1)
    _check(load().mppi_set_terrain_weights(ctrl.handle, w.ctypes.data_as(ctypes.c_void_p), w.shape[0]))


def terrain_weights(Yv, Yw, Fv, Fw, w_prev, gamma):
    """Eq. 4 on the host (exact); Fv, Fw (H, M).  Returns w (M,) float64."""
    Yv = np.ascontiguousarray(np.asarray(Yv, dtype=np.float64).reshape(-1))
    Yw = np.ascontiguousarray(np.asarray(Yw, dtype=np.float64).reshape(-1))
    Fv = np.ascontiguousarray(np.asarray(Fv, dtype=np.float64))
    Fw = np.ascontiguousarray(np.asarray(Fw, dtype=np.float64))
    wp = np.ascontiguousarray(np.asarray(w_prev, dtype=np.float64).reshape(-1))
    H, M = Fv.shape
    if Fw.shape != (H, M) or Yv.shape[0] != H or Yw.shape[0] != H or wp.shape[0] != M:
        raise ValueError("terrain_weights: inconsistent shapes")
    out = np.zeros(M)
    vp = ctypes.c_void_p
    _check(load().terrain_weights(Yv.ctypes.data_as(vp), Yw.ctypes.data_as(vp), Fv.ctypes.data_as(vp),
                                  Fw.ctypes.data_as(vp), H, M, wp.ctypes.data_as(vp), float(gamma),
                                  out.ctypes.data_as(vp)))
    return out


def mppi_step(ctrl: Ctrl, state, U_nom, U_new, weights=None, costs=None, stream=None):
    st = _f32(state).reshape(5)
    _check(load().mppi_step(ctrl.handle, st.ctypes.data_as(ctypes.c_void_p),
                            _dptr(U_nom, numel=2 * ctrl.T, name="U_nom"),
                            _dptr(U_new, numel=2 * ctrl.T, name="U_new"),
                            _dptr(weights, numel=ctrl.K, name="weights"),
                            _dptr(costs, numel=ctrl.K, name="costs"), _stream(stream)))


def mppi_step_host(ctrl: Ctrl, state, U_nom, U_new, weights=None, costs=None, stream=None):
    """mppi_step with every array on the host; returns once the outputs are there."""
    st = _f32(state).reshape(5)
    _check(load().mppi_step_host(ctrl.handle, st.ctypes.data_as(ctypes.c_void_p),
                                 _hptr(U_nom, 2 * ctrl.T, "U_nom"),
                                 _hptr(U_new, 2 * ctrl.T, "U_new", writable=True),
                                 _hptr(weights, ctrl.K, "weights", writable=True),
                                 _hptr(costs, ctrl.K, "costs", writable=True), _stream(stream)))


def mppi_rollout_trace(ctrl: Ctrl, state, U_nom, mu=None, sigma=None, stage=None, margins=None,
                       costs=None, stream=None):
    st = _f32(state).reshape(5)
    KT = ctrl.K * ctrl.T
    _check(load().mppi_rollout_trace(ctrl.handle, st.ctypes.data_as(ctypes.c_void_p),
                                     _dptr(U_nom, numel=2 * ctrl.T, name="U_nom"),
                                     _dptr(mu, numel=5 * KT, name="mu"),
                                     _dptr(sigma, numel=15 * KT, name="sigma"),
                                     _dptr(stage, numel=KT, name="stage"),
                                     _dptr(margins, numel=2 * KT, name="margins"),
                                     _dptr(costs, numel=ctrl.K, name="costs"), _stream(stream)))


def mppi_set_iteration(ctrl: Ctrl, it: int):
    _check(load().mppi_set_iteration(ctrl.handle, int(it)))


def mppi_get_iteration(ctrl: Ctrl) -> int:
    v = ctypes.c_uint64()
    _check(load().mppi_get_iteration(ctrl.handle, ctypes.byref(v)))
    return v.value


def mppi_nominal_sxy(ctrl: Ctrl, out, stream=None):
    _check(load().mppi_nominal_sxy(ctrl.handle, _dptr(out, numel=3 * ctrl.T, name="sxy"),
                                   _stream(stream)))


def mppi_rollout_kind(ctrl: Ctrl) -> int:
    """GPMPPI_KERNEL_* of the rollout kernel mppi_step runs for this controller."""
    v = ctypes.c_int32()
    _check(load().mppi_rollout_kind(ctrl.handle, ctypes.byref(v)))
    return v.value


def mppi_set_wait_limit(ctrl: Ctrl, ns: int, expire_first: bool = False):
    """Failure-detection hook of the FP32 rollout: limit (ns) of each bounded
    tile-copy wait and, with expire_first, a first wait that nothing completes."""
    _check(load().mppi_set_wait_limit(ctrl.handle, int(ns), 1 if expire_first else 0))


def mppi_set_profiling(ctrl: Ctrl, on: bool):
    _check(load().mppi_set_profiling(ctrl.handle, 1 if on else 0))


def mppi_last_profile(ctrl: Ctrl):
    """(rollout_ms, update_ms) of the last profiled mppi_step (waits for it)."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().mppi_last_profile(ctrl.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mppi_device_status(ctrl: Ctrl):
    """Raise if a rollout kernel reported a device-side failure (synchronises)."""
    _check(load().mppi_device_status(ctrl.handle))


def mppi_destroy(ctrl: Ctrl):
    if ctrl.handle:
        _check(load().mppi_destroy(ctrl.handle))
        ctrl.handle = None


def mppi_grad(ctrl: Ctrl, state, U_nom, slope=20.0, weights=None, J=None, dU=None, dl=None,
              want_dU=True, want_dl=True, stream=None):
    """Smoothed rollout cost J and its adjoint gradients dJ/dU (T,2) and
    dJ/dl (2,4) (see mppi_grad in the C header).  Returns (J, dU, dl) as CUDA
    tensors; dU / dl are None when not requested."""
    import torch
    dev = U_nom.device
    if J is None:
        J = torch.empty(1, dtype=torch.float32, device=dev)
    if want_dU and dU is None:
        dU = torch.empty(ctrl.T, 2, dtype=torch.float32, device=dev)
    if want_dl and dl is None:
        dl = torch.empty(2, 4, dtype=torch.float32, device=dev)
    if not want_dU:
        dU, dl = None, None
    if not want_dl:
        dl = None
    st = _f32(state).reshape(5)
    _check(load().mppi_grad(ctrl.handle, st.ctypes.data_as(ctypes.c_void_p),
                            _dptr(U_nom, torch.float32, 2 * ctrl.T, "U_nom"),
                            _dptr(weights, torch.float32, ctrl.K, "weights"), float(slope),
                            _dptr(J, torch.float32, 1, "J"),
                            _dptr(dU, torch.float32, 2 * ctrl.T, "dU"),
                            _dptr(dl, torch.float32, 8, "dl"), _stream(stream)))
    return J, dU, dl


def _make_autograd():
    import torch

    class SmoothedRolloutCost(torch.autograd.Function):
        """J(U, l) of mppi_grad as a differentiable op.  The adjoint kernel
        returns the gradients in the same pass as J, so forward computes them
        (only those whose inputs require grad) and backward scales them."""

        @staticmethod
        def forward(ctx, U, lengthscale, ctrl, state, slope, weights):
            need_u = ctx.needs_input_grad[0]
            need_l = ctx.needs_input_grad[1]
            J, dU, dl = mppi_grad(ctrl, state, U.detach().contiguous(), slope, weights,
                                  want_dU=need_u or need_l, want_dl=need_l)
            ctx.save_for_backward(dU if dU is not None else torch.zeros_like(U),
                                  dl if dl is not None else torch.zeros(2, 4, device=U.device))
            return J.reshape(())

        @staticmethod
        def backward(ctx, gJ):
            dU, dl = ctx.saved_tensors
            return gJ * dU, gJ * dl, None, None, None, None

    return SmoothedRolloutCost


_AUTOGRAD = None


def smoothed_rollout_cost(ctrl: Ctrl, state, U, lengthscale=None, slope=20.0, weights=None):
    """Differentiable smoothed chance-constrained rollout cost (torch scalar).

    U (T,2) CUDA tensor; lengthscale (2,4) CUDA tensor equal to the lengthscales
    the controller's GP was fitted with (refit and recreate the controller to
    move them), or None.  Gradients flow to whichever of U / lengthscale
    requires grad."""
    import torch
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    if lengthscale is None:
        lengthscale = torch.tensor([list(h.lengthscale) for h in ctrl.gp.hyper],
                                   dtype=torch.float32, device=U.device)
    elif ctrl.gp.hyper is not None:
        fitted = np.array([list(h.lengthscale) for h in ctrl.gp.hyper], dtype=np.float32)
        if not np.allclose(lengthscale.detach().cpu().numpy(), fitted, rtol=1e-6, atol=0):
            raise ValueError("lengthscale differs from the fitted GP's; refit the GP first")
    return _AUTOGRAD.apply(U, lengthscale, ctrl, state, float(slope), weights)


def mppi_update_noalloc(costs, u_tilde, U_nom, U_new, weights, K: int, T: int, lam: float,
                        stream=None):
    """Weights and control update with no device allocation (for callers that
    cannot allocate once running); u_tilde is (T, K, 2), step-major.  Every
    array is float32 on the current device (anything else raises ValueError
    before the library is called)."""
    import torch
    f32 = torch.float32
    for name, t in (("costs", costs), ("u_tilde", u_tilde), ("U_nom", U_nom), ("U_new", U_new),
                    ("weights", weights)):
        if t is not None and t.dtype != f32:
            raise ValueError(f"{name} must have dtype {f32}")
    _check(load().mppi_update_noalloc(_dptr(costs, f32, K, "costs"),
                                      _dptr(u_tilde, f32, 2 * K * T, "u_tilde"),
                                      _dptr(U_nom, f32, 2 * T, "U_nom"),
                                      _dptr(U_new, f32, 2 * T, "U_new"),
                                      _dptr(weights, f32, K, "weights"), K, T, float(lam),
                                      _stream(stream)))


def gpmppi_philox(seed: int, ctr, out, stream=None):
    M = ctr.numel() // 4
    _check(load().gpmppi_philox(int(seed) & 0xFFFFFFFFFFFFFFFF, _dptr(ctr, name="ctr"), M,
                                _dptr(out, numel=4 * M, name="out"), _stream(stream)))


def gpmppi_control_noise(seed: int, K: int, T: int, it: int, sigma, eps, stream=None):
    sg = (ctypes.c_float * 2)(float(sigma[0]), float(sigma[1]))
    _check(load().gpmppi_control_noise(int(seed) & 0xFFFFFFFFFFFFFFFF, K, T, int(it), sg,
                                       _dptr(eps, numel=2 * K * T, name="eps"), _stream(stream)))


def gpmppi_mma_selftest(fmt: int, A, B, D, variant: int = 0):
    """D = A B^T through the library's tcgen05 path (A: 128 x K, B: N x K 16-bit
    tensors viewed as int16/uint16, D: 128 x N float32)."""
    N, K = B.shape
    _check(load().gpmppi_mma_selftest(fmt, N, K, variant, _dptr(A, name="A"), _dptr(B, name="B"),
                                      _dptr(D, numel=128 * N, name="D")))


def gpmppi_alu_probe(kind: int, blocks: int, iters: int, out, stream=None):
    """Launch the throughput probe of one arithmetic unit (0: FP32 FMA, 1: packed
    FP32x2 FMA, 2: SFU ex2); blocks * 256 * iters * 16 operations."""
    _check(load().gpmppi_alu_probe(int(kind), int(blocks), int(iters),
                                   _dptr(out, numel=256 * blocks, name="out"), _stream(stream)))


class _DevArray:
    """A device pointer exposed through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr, shape, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _as_tensor(ptr, shape):
    import torch
    return torch.as_tensor(_DevArray(ptr, shape), device="cuda")


class Batch:
    """Owning wrapper of a gpmppi_batch handle (keeps its controllers alive).
    ``state[i]``, ``U_nom[i]``, ``U_new[i]``, ``weights[i]`` and ``costs[i]``
    are torch views of the batch's device buffers for controller i."""

    def __init__(self, handle, ctrls):
        self.handle, self.ctrls = handle, list(ctrls)
        self.state, self.U_nom, self.U_new, self.weights, self.costs = [], [], [], [], []
        for i, c in enumerate(self.ctrls):
            ptrs = [ctypes.c_void_p() for _ in range(5)]
            _check(load().mppi_batch_buffers(handle, i, *[ctypes.byref(p) for p in ptrs]))
            self.state.append(_as_tensor(ptrs[0].value, (5,)))
            self.U_nom.append(_as_tensor(ptrs[1].value, (c.T, 2)))
            self.U_new.append(_as_tensor(ptrs[2].value, (c.T, 2)))
            self.weights.append(_as_tensor(ptrs[3].value, (c.K,)))
            self.costs.append(_as_tensor(ptrs[4].value, (c.K,)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mppi_batch_destroy(self.handle)
            self.handle = None


def mppi_batch_create(ctrls) -> Batch:
    arr = (ctypes.c_void_p * len(ctrls))(*[c.handle for c in ctrls])
    h = ctypes.c_void_p()
    _check(load().mppi_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(ctrls), ctypes.byref(h)))
    return Batch(h.value, ctrls)


def mppi_batch_step(batch: Batch, stream=None):
    _check(load().mppi_batch_step(batch.handle, _stream(stream)))


def mppi_batch_graph(batch: Batch, stream=None):
    _check(load().mppi_batch_graph(batch.handle, _stream(stream)))


def mppi_batch_autotune(batch: Batch, stream=None) -> int:
    """Per-shape tile layouts and queue order from measured tile times;
    returns the number of controllers whose layout changed."""
    v = ctypes.c_int32()
    _check(load().mppi_batch_autotune(batch.handle, _stream(stream), ctypes.byref(v)))
    return v.value


def mppi_batch_layout(batch: Batch, i: int):
    """(producer threads per sample of controller i's tensor-core tiles (0 for
    FP32), time per tile in microseconds)."""
    r, t = ctypes.c_int32(), ctypes.c_float()
    _check(load().mppi_batch_layout(batch.handle, int(i), ctypes.byref(r), ctypes.byref(t)))
    return r.value, t.value


def mppi_batch_get_iteration(batch: Batch, i: int) -> int:
    v = ctypes.c_uint64()
    _check(load().mppi_batch_get_iteration(batch.handle, i, ctypes.byref(v)))
    return v.value


def mppi_batch_destroy(batch: Batch):
    if batch.handle:
        _check(load().mppi_batch_destroy(batch.handle))
        batch.handle = None
