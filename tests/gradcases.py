"""Small hand-built scenarios for the gradient of the smoothed rollout cost."""
import numpy as np

import scenarios as S


def tiny(shared=False):
    """K=2, T=2, N=2, one obstacle, straight lane: small enough to write the
    whole objective as one closed-form expression.  The start is off the lane
    centre, the noise small enough that no control leaves its box, and the
    obstacle and lane half-width chosen so that both sigmoids have slope."""
    sc = S.scenario("small", K=2, T=2, N=2, O=1, path="straight", sigma=(0.05, 0.05),
                    lane_half_width=0.25, seed=3)
    X = np.array([[0.9, 0.3, 1.1, 0.2], [1.3, -0.2, 0.8, 0.5]])
    Y = np.array([[0.05, -0.03], [-0.02, 0.04]])
    if shared:
        hyper = (S.Hyper((0.7, 0.6, 0.8, 0.9)), S.Hyper((0.7, 0.6, 0.8, 0.9)))
    else:
        hyper = (S.Hyper((0.7, 0.6, 0.8, 0.9)), S.Hyper((0.5, 0.9, 0.6, 0.7)))
    obst = np.array([[1.35, 0.45, 0.2]])
    x0 = np.array([1.0, 0.2, 0.3, 1.0, 0.5])
    U = np.array([[1.2, 0.3], [1.0, -0.2]])
    return sc.replace(X=X, Y=Y, hyper=hyper, obstacles=obst, x0=x0, U0=U)
