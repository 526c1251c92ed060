"""Philox4x32-10 counter-based RNG and Box-Muller normals (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Philox4x32 is defined in Salmon, Moraes, Dror, Shaw, "Parallel Random
Numbers: As Easy as 1, 2, 3" (SC'11): a 128-bit counter (four 32-bit words)
is mixed with a 64-bit key (two words) by R rounds of

    (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),
                         hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

with the Weyl key schedule k0 += W0, k1 += W1 between rounds.  The
multipliers and Weyl constants below are the ones published with the
generator; R = 10 is the recommended round count.

Draw assignment used by the controller (Alg. 1 Step 1 "Sample eps^s"):
key = (seed_lo, seed_hi), counter = (k, s, it_lo, it_hi) for time step k,
sample s and MPPI iteration it.  Words 0 and 1 of the output feed one
Box-Muller pair giving the (v_cmd, omega_cmd) perturbation of (s, k).
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: (..., 4) integers < 2**32; key: (..., 2) (broadcastable).
    Returns (..., 4) uint32.  Products are formed in uint64, which holds a
    32x32-bit product exactly.
    """
    ctr = np.asarray(ctr, dtype=np.uint64)
    key = np.asarray(key, dtype=np.uint64)
    c0, c1, c2, c3 = (ctr[..., i] for i in range(4))
    k0, k1 = key[..., 0], key[..., 1]
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    mask, sh = np.uint64(_MASK), np.uint64(32)
    w0, w1 = np.uint64(PHILOX_W0), np.uint64(PHILOX_W1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + w0) & mask
            k1 = (k1 + w1) & mask
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> sh) ^ c1 ^ k0, p1 & mask,
                          (p0 >> sh) ^ c3 ^ k1, p0 & mask)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniforms_from_words(w):
    """Map uint32 words to doubles in the open interval (0, 1): (w + 1/2) / 2^32."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * (2.0 ** -32)


def box_muller(u0, u1):
    """Standard-normal pair from two independent uniforms (Box & Muller, 1958)."""
    rad = np.sqrt(-2.0 * np.log(u0))
    ang = 2.0 * np.pi * u1
    return rad * np.cos(ang), rad * np.sin(ang)


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & _MASK, seed >> 32], dtype=np.uint64)


def control_noise(seed, k, samples, it, sigma):
    """Perturbation eps_k^s ~ N(0, diag(sigma^2)) of Alg. 1 Step 1.

    Returns (len(samples), 2) float64 for time step k and iteration it.
    """
    samples = np.asarray(samples, dtype=np.uint64)
    it = int(it)
    ctr = np.zeros(samples.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = np.uint64(k)
    ctr[..., 1] = samples
    ctr[..., 2] = np.uint64(it & _MASK)
    ctr[..., 3] = np.uint64((it >> 32) & _MASK)
    w = philox4x32_10(ctr, seed_key(seed))
    z0, z1 = box_muller(uniforms_from_words(w[..., 0]), uniforms_from_words(w[..., 1]))
    return np.stack([sigma[0] * z0, sigma[1] * z1], axis=-1)
