"""The GP-variance tolerance (1e-4 sigma_f^2 for FP32 and the FP16 hi/lo split,
1e-3 for the BF16 split) follows from the arithmetic: s = sigma_f^2 - |L^-1 k*|^2
(Sec. III-A) is evaluated here on the CPU in each of those arithmetics -
operands rounded to the format, products and sums in FP32 - and compared with
the FP64 oracle at cfg2's training set (N = 500), at random queries and at
queries next to training points, where |L^-1 k*|^2 nearly cancels sigma_f^2.
This is a numerics model of the tolerance, not of any kernel's summation
order."""
import numpy as np
import pytest

import oracle as O
import scenarios as S


def _queries(sc, rng):
    lo, hi = np.array([0.0, -1.5, 0.0, -1.5]), np.array([2.0, 1.5, 2.0, 1.5])
    far = lo + (hi - lo) * rng.random((48, 4))
    near = sc.X[rng.integers(0, sc.N, 48)] + 0.01 * rng.standard_normal((48, 4))
    return np.vstack([far, near])


def _split(x, dtype):
    """hi + lo with hi = rn(x) and lo = rn(x - hi) in a 16-bit format
    (BF16 emulated by rounding the FP32 significand to 8 bits)."""
    def rn(v):
        v = np.asarray(v, dtype=np.float32)
        if dtype == "fp16":
            return v.astype(np.float16).astype(np.float32)
        b = v.view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000          # round to nearest even
        return b.astype(np.uint32).view(np.float32)
    hi = rn(x)
    lo = rn(np.asarray(x, dtype=np.float32) - hi)
    return hi, lo


def _errors(fmt):
    sc = S.scenario("cfg2")
    f = O.gp_fit(sc.X, sc.Y, sc.hyper)[0]
    sf2 = f["signal_var"]
    Z = _queries(sc, np.random.default_rng(7))
    a = O.se_ard(Z, sc.X, f["lengthscale"], 1.0)                 # k* / sigma_f^2, (M, N)
    _, var64 = O.gp_predict([f, f], Z)
    s64 = var64[:, 0]
    W = f["Linv"].T                                                # V = a W (row form of L^-1 k*)
    if fmt == "fp32":
        V = a.astype(np.float32) @ W.astype(np.float32)
        q = np.sum(V * V, axis=1, dtype=np.float32) * np.float32(sf2 * sf2)
    else:
        cB = 2.0 ** np.floor(np.log2(16384.0 / np.max(np.abs(W))))
        Ah, Al = _split(a, fmt)
        Bh, Bl = _split(cB * W, fmt)
        V = Ah @ Bh + Al @ Bh + Ah @ Bl                             # FP32 products and sums
        q = np.sum(V * V, axis=1, dtype=np.float32) * np.float32((sf2 / cB) ** 2)
    s = np.maximum(0.0, sf2 - q.astype(np.float64))
    return np.max(np.abs(s - s64)) / sf2, np.min(s64) / sf2


@pytest.mark.parametrize("fmt,tol", [("fp32", 1e-4), ("fp16", 1e-4), ("bf16", 1e-3)])
def test_variance_error_within_declared_tolerance(fmt, tol):
    err, smallest = _errors(fmt)
    assert smallest < 0.05                 # the near-data queries do reach the cancellation regime
    assert err <= tol, (fmt, err)


def test_split_formats_are_ordered():
    # the BF16 split carries 16 significand bits, the FP16 split 22: its error is the larger
    assert _errors("bf16")[0] > _errors("fp16")[0]
