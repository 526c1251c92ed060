"""Seeded synthetic scenarios for the chance-constrained GP-MPPI rollout.

This module generates INPUTS only: GP training sets, obstacle fields,
reference paths, initial states and controller parameters.  It holds none
of the controller's arithmetic (no dynamics, GP algebra, costs or MPPI
update), so both the FP64 oracle and the CUDA path may take their inputs
from here without sharing any of the method's code.

The paper's dataset (Rabiee et al., the 6 km Jackal log used in Sec. V-A)
is not available, so a synthetic residual stands in for it with the same
shape as the paper's GP: 4-D inputs (v, omega, v_cmd, omega_cmd) inside the
robot's operating box and two residual outputs (delta_v, delta_omega).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

# Operating box of the GP inputs (v, omega, v_cmd, omega_cmd); it is also
# the control box [u_min, u_max] for (v_cmd, omega_cmd).
GP_INPUT_LO = np.array([0.0, -1.5, 0.0, -1.5])
GP_INPUT_HI = np.array([2.0, 1.5, 2.0, 1.5])


@dataclass
class Params:
    """Controller parameters (Alg. 1 inputs plus the readings of the paper).

    Field names follow the paper: alpha are the tracking weights of Eq. 11,
    beta the avoidance weights of Eq. 12, p_x the chance level of Eq. 7,
    lam the MPPI temperature, sigma the std of Sigma_sim.
    """

    K: int = 256                      # number of MPPI samples (S in Alg. 1)
    T: int = 20                       # horizon (N in Eq. 5 / Alg. 1)
    dt: float = 0.05
    tau_v: float = 0.3
    tau_w: float = 0.2
    sigma: tuple = (0.5, 0.8)        # control-noise std (v_cmd, omega_cmd)
    lam: float = 1.0
    p_x: float = 0.95
    u_min: tuple = (0.0, -1.5)
    u_max: tuple = (2.0, 1.5)
    alpha: tuple = (1.0, 1.0, 0.0, 1.0, 0.5)
    beta: tuple = (0.0, 1.0, 0.0, 0.0)
    P_lane: float = 100.0
    P_coll: float = 1000.0
    lane_half_width: float = 1.0
    v_desired: float = 1.5
    seed: int = 0
    variance_mode: int = 0            # 0 = per sample, 1 = nominal (Alg. 1 Step 2)
    precision: int = 0                # 0 = FP32, 1 = BF16 hi/lo split, 2 = FP16 hi/lo split
    goal: tuple = (0.0, 0.0)          # goal position of the stage and terminal terms (Eq. 12)
    goal_radius: float = 0.5          # the terminal term fires when the final mean is farther
    P_goal: float = 100.0             # penalty multiplying the terminal indicator


@dataclass
class Hyper:
    """SE-ARD hyper-parameters of one GP output."""

    lengthscale: tuple = (0.5, 0.5, 0.5, 0.5)
    signal_var: float = 0.1
    noise_var: float = 1e-4


@dataclass
class Scenario:
    name: str
    params: Params
    X: np.ndarray           # (N, 4) float64 GP inputs
    Y: np.ndarray           # (N, 2) float64 GP targets (delta_v, delta_omega)
    hyper: tuple            # (Hyper, Hyper) for the two outputs
    obstacles: np.ndarray   # (O, 3) float64: cx, cy, radius
    path: np.ndarray        # (P, 2) float64 polyline of the lane centre
    x0: np.ndarray          # (5,) initial state X, Y, theta, v, omega
    U0: np.ndarray          # (T, 2) initial nominal control sequence
    meta: dict = field(default_factory=dict)
    # terrain ensemble (Eq. 3): M training sets and hyper-parameter pairs, and
    # the weights w_i; None for the single GP above
    terrains: list = None   # [(X_i, Y_i, (Hyper, Hyper)), ...]
    terrain_w: tuple = None

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    def replace(self, **kw) -> "Scenario":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# synthetic ground truth (stand-in for the paper's terrain dataset)
# --------------------------------------------------------------------------

def true_residual(v, w, v_cmd, w_cmd):
    """Synthetic terrain residual: delta_v = -0.1 v |w|, delta_w = -0.2 w v.

    This is the simulated world the controller does not know; the GP is
    trained on noisy samples of it and the closed-loop plant adds it.
    """
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    return np.stack([-0.1 * v * np.abs(w), -0.2 * w * v], axis=-1)


def gp_training_set(rng: np.random.Generator, N: int):
    """N points uniform in the operating box with noisy residual targets."""
    X = GP_INPUT_LO + (GP_INPUT_HI - GP_INPUT_LO) * rng.random((N, 4))
    Y = true_residual(X[:, 0], X[:, 1], X[:, 2], X[:, 3])
    Y = Y + np.sqrt(1e-4) * rng.standard_normal((N, 2))
    return X, Y


# --------------------------------------------------------------------------
# reference paths
# --------------------------------------------------------------------------

def path_straight(length: float = 20.0) -> np.ndarray:
    return np.array([[0.0, 0.0], [length, 0.0]])


def path_figure_eight(a: float = 5.0, P: int = 512) -> np.ndarray:
    """Lemniscate of Gerono x = a sin t, y = a sin t cos t, closed (last = first)."""
    t = np.linspace(0.0, 2.0 * np.pi, P)
    pts = np.stack([a * np.sin(t), a * np.sin(t) * np.cos(t)], axis=1)
    pts[-1] = pts[0]
    return pts


def path_sinusoid(A: float = 2.0, wavelength: float = 10.0, length: float = 40.0,
                  P: int = 512) -> np.ndarray:
    x = np.linspace(0.0, length, P)
    return np.stack([x, A * np.sin(2.0 * np.pi * x / wavelength)], axis=1)


def initial_state(path: np.ndarray, v0: float = 1.0) -> np.ndarray:
    """Start on the first path vertex, heading along the first segment."""
    d = path[1] - path[0]
    return np.array([path[0, 0], path[0, 1], np.arctan2(d[1], d[0]), v0, 0.0])


def obstacles_uniform(rng, O, box, r_lo, r_hi, path=None, clearance=None):
    """O circles with centres uniform in box=(xlo, xhi, ylo, yhi).

    When ``clearance`` is given, centres closer than that to any path vertex
    are redrawn (the vertices are dense, so this keeps centres off the lane
    centre without using the controller's own distance arithmetic).
    """
    out = []
    while len(out) < O:
        c = np.array([box[0] + (box[1] - box[0]) * rng.random(),
                      box[2] + (box[3] - box[2]) * rng.random()])
        r = r_lo if r_hi == r_lo else r_lo + (r_hi - r_lo) * rng.random()
        if clearance is not None and path is not None:
            if np.min(np.hypot(path[:, 0] - c[0], path[:, 1] - c[1])) < clearance:
                continue
        out.append([c[0], c[1], r])
    return np.array(out, dtype=np.float64).reshape(O, 3)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def scenario(name: str, **overrides) -> Scenario:
    """Build one of the named workloads.

    cfg1: K=256, T=20, N=50, 4 obstacles r=0.3 in [0,10]x[-5,5], straight path, seed 0.
    cfg2: K=4096, T=50, N=500, 16 obstacles r in [0.2,0.6], figure-eight a=5, seed 1.
    cfg3: K=16384, T=100, N=2048, 64 obstacles, figure-eight, BF16 split, seed 1.
    cfg4: K=4096, T=50, N=1000, 16 obstacles, figure-eight, seed 1.
    small: a fast case spanning several tiles with ragged tails (K=77, T=7, N=45).
    ``overrides`` replace Params fields or K/T/N/O/seed before generation.
    """
    seed = overrides.pop("seed", None)
    if name == "cfg1":
        p = Params(K=256, T=20, seed=0)
        N, O, kind = 50, 4, "straight"
    elif name == "cfg2":
        p = Params(K=4096, T=50, seed=1)
        N, O, kind = 500, 16, "eight"
    elif name == "cfg3":
        p = Params(K=16384, T=100, seed=1, precision=1)
        N, O, kind = 2048, 64, "eight"
    elif name == "cfg4":
        p = Params(K=4096, T=50, seed=1)
        N, O, kind = 1000, 16, "eight"
    elif name == "small":
        p = Params(K=77, T=7, seed=5)
        N, O, kind = 45, 6, "eight"
    else:
        raise ValueError(f"unknown scenario {name!r}")
    if seed is not None:
        p.seed = int(seed)
    N = int(overrides.pop("N", N))
    O = int(overrides.pop("O", O))
    kind = overrides.pop("path", kind)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise ValueError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    rng = np.random.Generator(np.random.PCG64(p.seed))
    if kind == "straight":
        path = path_straight()
    elif kind == "eight":
        path = path_figure_eight(5.0, 512)
    elif kind == "sine":
        path = path_sinusoid()
    else:
        raise ValueError(kind)
    # training set first so that it does not depend on the obstacle draw
    X, Y = gp_training_set(rng, N)
    if name == "cfg1":
        obst = obstacles_uniform(rng, O, (0.0, 10.0, -5.0, 5.0), 0.3, 0.3)
    elif name == "cfg3":
        obst = obstacles_uniform(rng, O, (-8.0, 8.0, -4.0, 4.0), 0.2, 0.6, path, 0.3)
    else:
        obst = obstacles_uniform(rng, O, (-6.0, 6.0, -3.0, 3.0), 0.2, 0.6, path, 0.3)
    x0 = initial_state(path)
    U0 = np.tile(np.array([p.v_desired, 0.0]), (p.T, 1))
    return Scenario(name=name, params=p, X=X, Y=Y, hyper=(Hyper(), Hyper()),
                    obstacles=obst, path=path, x0=x0, U0=U0, meta={"path": kind})


# --------------------------------------------------------------------------
# terrain ensemble (Eq. 3): stand-ins for the paper's grass, asphalt and tile
# --------------------------------------------------------------------------

TERRAIN_COEF = (      # (a, b, c): delta_v = -a v |w| - c v, delta_w = -b w v
    (0.15, 0.30, 0.05),
    (0.05, 0.10, 0.00),
    (0.10, 0.20, 0.02),
)
TERRAIN_LENGTHSCALE = (0.5, 0.6, 0.45)
TERRAIN_SIGNAL_VAR = (0.1, 0.08, 0.12)


def terrain_residual(i, v, w, v_cmd, w_cmd):
    """Synthetic residual of terrain i (the controller only sees GP fits of it)."""
    a, b, c = TERRAIN_COEF[i % len(TERRAIN_COEF)]
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    return np.stack([-a * v * np.abs(w) - c * v, -b * w * v], axis=-1)


def terrain_scenario(name: str = "cfg2", M: int = 3, N: int = None, w=None, **overrides) -> Scenario:
    """The named workload with its single GP replaced by M terrain GPs (N
    points each, own hyper-parameters shared by the two outputs of a terrain)
    mixed with weights w (Eq. 3)."""
    sc = scenario(name, **overrides)
    N = sc.N if N is None else int(N)
    rng = np.random.Generator(np.random.PCG64(7_000 + sc.params.seed))
    terrains = []
    for i in range(M):
        X = GP_INPUT_LO + (GP_INPUT_HI - GP_INPUT_LO) * rng.random((N, 4))
        Y = terrain_residual(i, X[:, 0], X[:, 1], X[:, 2], X[:, 3])
        Y = Y + np.sqrt(1e-4) * rng.standard_normal((N, 2))
        ell = TERRAIN_LENGTHSCALE[i % 3]
        h = Hyper((ell,) * 4, TERRAIN_SIGNAL_VAR[i % 3], 1e-4)
        terrains.append((X, Y, (h, Hyper(h.lengthscale, h.signal_var, h.noise_var))))
    if w is None:
        w = (0.5, 0.3, 0.2)[:M] if M <= 3 else tuple([1.0 / M] * M)
        w = tuple(np.asarray(w) / np.sum(w))
    return sc.replace(name=f"{name}-terrain{M}", terrains=terrains, terrain_w=tuple(float(x) for x in w))


def batched_scenarios(B: int = 64, first_seed: int = 0):
    """Heterogeneous controllers: K in [1024,16384], T in [20,100], N in [200,4096],
    4..64 obstacles, alternating sinusoid / figure-eight paths; seeds first_seed.."""
    out = []
    for b in range(B):
        seed = first_seed + b
        rng = np.random.Generator(np.random.PCG64(10_000 + seed))
        K = int(rng.integers(1024, 16385))
        T = int(rng.integers(20, 101))
        N = int(rng.integers(200, 4097))
        O = int(rng.integers(4, 65))
        kind = "sine" if b % 2 == 0 else "eight"
        out.append(scenario("cfg2", seed=seed, K=K, T=T, N=N, O=O, path=kind))
    return out
