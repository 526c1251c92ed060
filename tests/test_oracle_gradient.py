"""Pins for the smoothed objective and its FP64 finite-difference gradient.

The smoothed cost replaces the indicators of Eq. 11-12 by sigmoids; the
gradient is central differences.  Pinned by (1) the limits of the sigmoid
(slope -> infinity gives the indicator cost, slope -> 0 gives half of each
penalty), (2) the symbolic derivative of a tiny case written out as one
closed-form expression (sympy differentiates it; the oracle differences
numerically), including the lengthscales of two GPs with different
hyper-parameters, and (3) Richardson consistency of the differences.
"""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gradcases import tiny


def _margins_clear(ro, eps):
    lm, om = ro["lane_margin"], ro["obs_margin"]
    return np.all(np.abs(lm) > eps, axis=1) & np.all(np.abs(om) > eps, axis=1)


def test_sigmoid_limits():
    sc = S.scenario("small")
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    U = sc.U0
    hard = O.rollout(sc, fits, sc.x0, U, 0)
    steep = O.rollout(sc, fits, sc.x0, U, 0, slope=1e9)
    ok = _margins_clear(hard, 1e-6)
    assert ok.sum() > 0.8 * sc.params.K
    np.testing.assert_allclose(steep["costs"][ok], hard["costs"][ok], rtol=1e-12, atol=1e-9)
    # slope -> 0: every sigmoid is 1/2
    flat = O.rollout(sc, fits, sc.x0, U, 0, slope=1e-12)
    P = sc.params
    T = P.T
    no_pen = sc.params.__class__(**{**P.__dict__, "P_lane": 0.0, "P_coll": 0.0})
    base = O.rollout(sc.replace(params=no_pen), fits, sc.x0, U, 0, slope=1e-12)
    extra = 0.5 * (P.alpha[3] * P.P_lane * sum(0.9 ** k for k in range(T)) + P.beta[1] * P.P_coll * T)
    np.testing.assert_allclose(flat["costs"] - base["costs"], extra, rtol=1e-9)


def _symbolic_objective(sc, slope):
    """The tiny case as a sympy expression in U (4 symbols) and l (8)."""
    sp = pytest.importorskip("sympy")
    P = sc.params
    u = sp.symbols("u0:4")
    ls = sp.symbols("l0:8")
    sf2 = [sp.Float(h.signal_var) for h in sc.hyper]
    sn2 = [sp.Float(h.noise_var) for h in sc.hyper]
    X = [[sp.Float(v) for v in row] for row in sc.X]

    def kern(a, b, o):
        return sf2[o] * sp.exp(-sp.Rational(1, 2) * sum(((a[d] - b[d]) / ls[4 * o + d]) ** 2 for d in range(4)))

    gps = []
    for o in range(2):
        Kxx = sp.Matrix(2, 2, lambda i, j: kern(X[i], X[j], o) + (sn2[o] if i == j else 0))
        Kinv = Kxx.inv()
        alpha = Kinv * sp.Matrix([sp.Float(sc.Y[0, o]), sp.Float(sc.Y[1, o])])
        gps.append((Kinv, alpha))

    def gp(z, o):
        Kinv, alpha = gps[o]
        ks = sp.Matrix([kern(z, X[0], o), kern(z, X[1], o)])
        return (ks.T * alpha)[0], sf2[o] - (ks.T * Kinv * ks)[0]

    sq_chi2, phi = O.mppi.tightening_constants(P.p_x)
    dt, tv, tw = sp.Float(P.dt), sp.Float(P.tau_v), sp.Float(P.tau_w)
    cx, cy, R = (sp.Float(v) for v in sc.obstacles[0])
    a, b = P.alpha, P.beta
    r = sp.Float(P.lane_half_width)
    sig = lambda x: 1 / (1 + sp.exp(-x))
    J = 0
    for s in range(P.K):
        X_, Y_, th, v, w = (sp.Float(x) for x in sc.x0)
        Sig = sp.zeros(5, 5)
        for k in range(P.T):
            eps = O.control_noise(P.seed, k, np.array([s]), 0, P.sigma)[0]
            ut = (u[2 * k] + sp.Float(eps[0]), u[2 * k + 1] + sp.Float(eps[1]))
            z = (v, w, ut[0], ut[1])
            (mv, sv), (mw, sw) = gp(z, 0), gp(z, 1)
            A = sp.Matrix([[1, 0, -dt * v * sp.sin(th), dt * sp.cos(th), 0],
                           [0, 1, dt * v * sp.cos(th), dt * sp.sin(th), 0],
                           [0, 0, 1, 0, dt],
                           [0, 0, 0, 1 - dt / tv, 0],
                           [0, 0, 0, 0, 1 - dt / tw]])
            X_, Y_, th, v, w = (X_ + dt * v * sp.cos(th), Y_ + dt * v * sp.sin(th), th + dt * w,
                                v + dt / tv * (ut[0] - v) + mv, w + dt / tw * (ut[1] - w) + mw)
            Sig = A * Sig * A.T + sp.diag(0, 0, 0, sv, sw)
            sxx, sxy, syy = Sig[0, 0], Sig[0, 1], Sig[1, 1]
            lam = (sxx + syy) / 2 + sp.sqrt(((sxx - syy) / 2) ** 2 + sxy ** 2)
            e = sp.sqrt(Y_ ** 2)                 # straight lane along the x axis
            rbar = r - sp.Float(sq_chi2) * sp.sqrt(lam)
            dx, dy = X_ - cx, Y_ - cy
            rho = sp.sqrt(dx ** 2 + dy ** 2)
            nx, ny = dx / rho, dy / rho
            dbar = rho - R - sp.Float(phi) * sp.sqrt(nx * nx * sxx + 2 * nx * ny * sxy + ny * ny * syy)
            trC = sv + sw
            J += (a[0] * trC + a[1] * e / r + a[3] * P.P_lane * sp.Float(0.9) ** k * sig(slope * (e - rbar))
                  + a[4] * (P.v_desired - v) ** 2 + b[0] * trC + b[1] * P.P_coll * sig(-slope * dbar))
    return J / P.K, u, ls


def test_fd_gradient_matches_symbolic():
    sp = pytest.importorskip("sympy")
    sc = tiny(shared=False)
    slope = 20.0
    Jsym, u, ls = _symbolic_objective(sc, slope)
    vals = {**{u[i]: sc.U0.reshape(-1)[i] for i in range(4)},
            **{ls[4 * o + d]: sc.hyper[o].lengthscale[d] for o in range(2) for d in range(4)}}
    syms = list(u) + list(ls)
    f = sp.lambdify(syms, [Jsym] + [sp.diff(Jsym, x) for x in syms], "numpy", cse=True)
    out = np.array(f(*[vals[x] for x in syms]), dtype=np.float64)
    J_ref, g_ref = out[0], out[1:]
    J, ro = O.objective(sc, sc.hyper, sc.x0, sc.U0, 0, None, slope)
    assert np.all(ro["u_tilde"] > np.array(sc.params.u_min)) and np.all(ro["u_tilde"] < np.array(sc.params.u_max))
    assert J == pytest.approx(J_ref, rel=1e-12)
    gU, gL = O.fd_gradient(sc, sc.hyper, sc.x0, sc.U0, 0, None, slope)
    g = np.concatenate([gU.reshape(-1), gL.reshape(-1)])
    # every component carries signal in this case
    assert np.all(np.abs(g_ref) > 1e-4)
    np.testing.assert_allclose(g, g_ref, rtol=2e-6, atol=1e-8 * np.max(np.abs(g_ref)))


def test_fd_richardson_consistency():
    sc = S.scenario("small", K=16, T=5, N=20)
    U = sc.U0 + 0.1
    g1, l1 = O.fd_gradient(sc, sc.hyper, sc.x0, U, 0, None, 20.0, h_u=1e-4, h_l=1e-4)
    g2, l2 = O.fd_gradient(sc, sc.hyper, sc.x0, U, 0, None, 20.0, h_u=5e-5, h_l=5e-5)
    scale = max(np.max(np.abs(g1)), np.max(np.abs(l1)))
    # central differences: error O(h^2), so halving h changes the result by far less than h
    assert np.max(np.abs(g1 - g2)) < 1e-5 * scale
    assert np.max(np.abs(l1 - l2)) < 1e-5 * scale
