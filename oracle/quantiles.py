"""Quantile functions used by the constraint tightening (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. 14 needs chi^2_2(p_x), the p_x quantile of a chi-squared variable with
two degrees of freedom; that distribution is exponential with mean 2, so its
quantile is -2 ln(1 - p).  Eq. 16 needs Phi^{-1}(p_x), the standard-normal
quantile; it is found here by bisection on Phi(x) = erfc(-x/sqrt 2)/2, which
converges to the double nearest the root (no rational approximation).
"""
from __future__ import annotations

import math


def chi2_2_quantile(p: float) -> float:
    if not (0.0 < p < 1.0):
        raise ValueError("p must lie in (0, 1)")
    return -2.0 * math.log1p(-p)


def normal_cdf(x: float) -> float:
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def normal_quantile(p: float) -> float:
    """Phi^-1(p) by bisection.  For p > 1/2 the search runs on the upper tail
    erfc(x/sqrt 2)/2 = 1 - p, which keeps full relative precision near 1."""
    if not (0.0 < p < 1.0):
        raise ValueError("p must lie in (0, 1)")
    if p > 0.5:
        q = 1.0 - p
        f = lambda x: 0.5 * math.erfc(x / math.sqrt(2.0)) > q   # noqa: E731  (x below root)
    else:
        f = lambda x: normal_cdf(x) < p                         # noqa: E731
    lo, hi = -40.0, 40.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if f(mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
