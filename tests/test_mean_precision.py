"""The GP mean k*.alpha (Sec. III-A) is a long sum of terms of both signs
that largely cancel (|alpha_j| far above the mean it produces), so its FP32
rounding error scales with sum |k_j alpha_j|.  A CPU model at cfg2's training
set: the compensated (Neumaier) sum of 16-point chunk partials, as the
kernels accumulate it, against a plain sequential FP32 sum and against FP16
hi/lo split products (the alternative of putting alpha into the tensor-core
contraction as extra columns), each compared with FP64."""
import numpy as np

import oracle as O
import scenarios as S
from test_variance_tolerance import _queries, _split


def _mean_errors(j):
    sc = S.scenario("cfg2")
    f = O.gp_fit(sc.X, sc.Y, sc.hyper)[j]
    sf2, al = f["signal_var"], f["alpha"]
    a = O.se_ard(_queries(sc, np.random.default_rng(7)), sc.X, f["lengthscale"], 1.0)
    m64 = sf2 * (a @ al)
    a32, al32 = a.astype(np.float32), al.astype(np.float32)
    M, N = a.shape
    plain = np.zeros(M, np.float32)
    for i in range(N):
        plain = plain + a32[:, i] * al32[i]
    s, c = np.zeros(M, np.float32), np.zeros(M, np.float32)
    for c0 in range(0, N, 16):
        pe, po = np.zeros(M, np.float32), np.zeros(M, np.float32)
        for q in range(c0, min(N, c0 + 16), 2):
            pe = pe + a32[:, q] * al32[q]
            if q + 1 < N:
                po = po + a32[:, q + 1] * al32[q + 1]
        x = pe + po
        t = s + x
        c = c + np.where(np.abs(s) >= np.abs(x), (s - t) + x, (x - t) + s)
        s = t
    cA = 2.0 ** np.floor(np.log2(16384.0 / np.max(np.abs(al))))
    Ah, Al = _split(a, "fp16")
    Bh, Bl = _split(cA * al, "fp16")
    split = (Ah @ Bh + Al @ Bh + Ah @ Bl).astype(np.float64) * (sf2 / cA)
    err = lambda m: float(np.max(np.abs(m - m64)))
    return err(sf2 * plain.astype(np.float64)), err(sf2 * (s + c).astype(np.float64)), err(split), \
        float(np.max(np.abs(al))), float(np.max(np.abs(m64)))


def test_alpha_dwarfs_the_mean():
    for j in range(2):
        *_, amax, mmax = _mean_errors(j)
        assert amax > 50 * mmax


def test_compensated_sum_is_the_most_accurate():
    for j in range(2):
        plain, comp, split, *_ = _mean_errors(j)
        assert comp <= 1e-6
        assert comp < split < plain
