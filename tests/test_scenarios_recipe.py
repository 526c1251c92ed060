"""The seeded synthetic workloads match their stated recipe (sizes, input
ranges, hyper-parameters, obstacle radii and clearance, path), so the
benchmark's configuration is the documented one.  The inputs stand in for
the paper's dataset (Sec. V-A), which is not available."""
import numpy as np
import pytest

import scenarios as S

SIZES = {  # K, T, N, obstacles, path vertices
    "cfg1": (256, 20, 50, 4, 2),
    "cfg2": (4096, 50, 500, 16, 512),
    "cfg3": (16384, 100, 2048, 64, 512),
    "cfg4": (4096, 50, 1000, 16, 512),
    "small": (77, 7, 45, 6, 512),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_sizes_inputs_and_hypers(name):
    sc = S.scenario(name)
    K, T, N, O, P = SIZES[name]
    assert (sc.params.K, sc.params.T, sc.N) == (K, T, N)
    assert sc.obstacles.shape == (O, 3) and sc.path.shape == (P, 2)
    # GP inputs (v, omega, v_cmd, omega_cmd) uniform in [0,2] x [-1.5,1.5] x [0,2] x [-1.5,1.5]
    assert sc.X.shape == (N, 4)
    lo, hi = np.array([0.0, -1.5, 0.0, -1.5]), np.array([2.0, 1.5, 2.0, 1.5])
    assert np.all(sc.X >= lo) and np.all(sc.X <= hi)
    for h in sc.hyper:
        assert tuple(h.lengthscale) == (0.5, 0.5, 0.5, 0.5)
        assert (h.signal_var, h.noise_var) == (0.1, 1e-4)


def test_cfg2_targets_follow_the_synthetic_residual():
    # dv = -0.1 v |w| and dw = -0.2 w v plus noise of variance 1e-4
    sc = S.scenario("cfg2")
    v, w = sc.X[:, 0], sc.X[:, 1]
    r_v = sc.Y[:, 0] - (-0.1 * v * np.abs(w))
    r_w = sc.Y[:, 1] - (-0.2 * w * v)
    for r in (r_v, r_w):
        assert abs(np.mean(r)) < 3e-3 and 0.005 < np.std(r) < 0.015


def test_cfg2_obstacles_and_seed():
    sc = S.scenario("cfg2")
    r = sc.obstacles[:, 2]
    assert np.all((r >= 0.2) & (r <= 0.6))
    c = sc.obstacles[:, :2]
    assert np.all(np.abs(c[:, 0]) <= 6.0) and np.all(np.abs(c[:, 1]) <= 3.0)
    d = np.min(np.linalg.norm(c[:, None, :] - sc.path[None, :, :], axis=2), axis=1)
    assert np.all(d >= 0.3)                       # clear of every path vertex
    again = S.scenario("cfg2")
    assert np.array_equal(again.X, sc.X) and np.array_equal(again.obstacles, sc.obstacles)
