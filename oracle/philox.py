"""Counter-based random numbers for the oracle (test infrastructure only).

This module is part of the CPU oracle.  Only the tests, the smoke check and the
bench's CPU-baseline leg may import it; the GPU product path never does.

AeroSketch draws two kinds of random matrices (Algorithm 1: the power-iteration
start vector x^(0) ~ N(0, I); Algorithm 2: the Gaussian test matrix Pi).  So that
the GPU path and this oracle draw the *same* numbers without sharing code, both
sides implement one published generator from its definition:

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC'11): a 4x64-bit counter, a 2x64-bit key, ten rounds of
  (hi, lo) = M * x multiplications with key bumps by the Weyl constants.
* uniform u = ((w >> 12) + 0.5) * 2^-52, exactly representable and strictly
  inside (0, 1) (with 53 bits the top word would round to 1.0);
* Gaussians by the Box-Muller transform: from the 4 words of one counter block,
  (z0, z1) = sqrt(-2 ln u0) * (cos 2 pi u1, sin 2 pi u1) and
  (z2, z3) = sqrt(-2 ln u2) * (cos 2 pi u3, sin 2 pi u3).

Counter layout (a reading, the paper fixes no generator):
    counter = (purpose, timestamp i, sub-index j, element e >> 2),
    key     = (seed, stream_id),
and element e of a matrix filled row-major takes lane e & 3 of its block.
Purposes used by the method: 3 = power-iteration start vector (Algorithm 1),
4 = simultaneous-iteration test matrix Pi (Algorithm 2, j = doubling step).

Pinned against numpy.random.Philox (an independent implementation of the same
published generator) in tests/test_oracle_philox.py.
"""
from __future__ import annotations

import numpy as np

PURPOSE_PI_START = 3   # Algorithm 1, x^(0)
PURPOSE_SI_TEST = 4    # Algorithm 2, Pi

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a: np.uint64, b: np.ndarray):
    """Full 64x64 -> 128-bit product, returned as (high word, low word)."""
    b = b.astype(np.uint64, copy=False)
    a0 = np.uint64(int(a) & 0xFFFFFFFF)
    a1 = np.uint64(int(a) >> 32)
    b0 = b & _LO32
    b1 = b >> _S32
    with np.errstate(over="ignore"):
        p00 = a0 * b0
        p01 = a0 * b1
        p10 = a1 * b0
        p11 = a1 * b1
        mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
        hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
        lo = np.uint64(a) * b
    return hi, lo


def philox4x64_10(counters: np.ndarray, key) -> np.ndarray:
    """Philox4x64 with 10 rounds.  counters: (N, 4) uint64, key: 2 words."""
    c = np.asarray(counters, dtype=np.uint64).reshape(-1, 4)
    x0, x1, x2, x3 = (c[:, t].copy() for t in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFFFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint64(k0 + _W0)
                k1 = np.uint64(k1 + _W1)
            hi0, lo0 = _mulhilo64(_M0, x0)
            hi1, lo1 = _mulhilo64(_M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=1)


def uniform53(words: np.ndarray) -> np.ndarray:
    """Map 64-bit words to doubles strictly inside (0, 1)."""
    w = np.asarray(words, dtype=np.uint64)
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussians(seed: int, stream_id: int, purpose: int, i: int, j: int, n: int) -> np.ndarray:
    """n standard normals for counter (purpose, i, j, .) under key (seed, stream_id).

    Element e comes from counter block e >> 2, lane e & 3 (Box-Muller pairs
    (0, 1) and (2, 3) of that block)."""
    nb = (n + 3) // 4
    ctr = np.zeros((nb, 4), dtype=np.uint64)
    ctr[:, 0] = np.uint64(purpose)
    ctr[:, 1] = np.uint64(i)
    ctr[:, 2] = np.uint64(j)
    ctr[:, 3] = np.arange(nb, dtype=np.uint64)
    w = philox4x64_10(ctr, (seed, stream_id))
    u = uniform53(w)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.empty((nb, 4), dtype=np.float64)
    z[:, 0] = r01 * np.cos(2.0 * np.pi * u[:, 1])
    z[:, 1] = r01 * np.sin(2.0 * np.pi * u[:, 1])
    z[:, 2] = r23 * np.cos(2.0 * np.pi * u[:, 3])
    z[:, 3] = r23 * np.sin(2.0 * np.pi * u[:, 3])
    return z.reshape(-1)[:n]
