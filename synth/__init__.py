"""Seeded synthetic row streams shared by the tests, the bench and the oracle.

This module only draws input data; it holds none of the sketching arithmetic.
The recipe stands in for the paper's "Random Noisy" workload (Section 5.1.3:
low-rank signal with a decaying spectrum plus Gaussian noise):

    rows = g diag(sigma) V^T + eta,
    g ~ N(0, 1)^{n x r},  V = Q factor of a d x r Gaussian (Householder QR,
    diag(R) > 0),  eta ~ N(0, noise^2)^{n x d},

generated in FP64 with numpy's Philox bit generator and rounded to FP32, so
both the GPU path and the oracle consume the identical FP32 bytes.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


def basis(d: int, r: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    """Random orthonormal d x r basis (Q of a Gaussian matrix, diag(R) > 0)."""
    g = _rng(seed, 1_000_000 + stream).standard_normal((d, r))
    q, rr = np.linalg.qr(g)
    return q * np.sign(np.diag(rr))[None, :]


def spectrum(kind: str, r: int) -> np.ndarray:
    if kind == "geometric":          # sigma_i = 10 * 0.9^i, i = 0..r-1
        return 10.0 * 0.9 ** np.arange(r)
    if kind == "powerlaw":           # sigma_i = 1 / i, i = 1..r
        return 1.0 / np.arange(1, r + 1)
    raise ValueError(kind)


def low_rank_noisy(n: int, d: int, r: int, sigma: np.ndarray, noise: float = 0.01,
                   seed: int = 0, stream: int = 0, start: int = 0,
                   V: np.ndarray | None = None, chunk: int = 4096) -> np.ndarray:
    """Rows start..start+n-1 of the stream, FP32, C-contiguous (n x d).

    Rows are drawn in chunks of `chunk` rows keyed by chunk index, so any
    window of the stream is reproducible without drawing the rows before it
    (streams with another chunk size are other streams)."""
    if V is None:
        V = basis(d, r, seed, stream)
    out = np.empty((n, d), dtype=np.float32)
    c0, c1 = start // chunk, (start + n + chunk - 1) // chunk
    for c in range(c0, c1):
        rng = _rng(seed, (stream << 32) + c)
        g = rng.standard_normal((chunk, r))
        eta = rng.standard_normal((chunk, d)) * noise
        blk = (g * sigma[None, :]) @ V.T + eta
        lo, hi = max(start, c * chunk), min(start + n, (c + 1) * chunk)
        out[lo - start:hi - start] = blk[lo - c * chunk:hi - c * chunk]
    return out


def givens_sweep(V: np.ndarray, seed: int, k: int) -> np.ndarray:
    """G_k V for the k-th sweep of Givens rotations on the coordinate pairs
    (j, j+1), j = 0 .. d-2 in order, angles uniform on [0, 2 pi) from a stream
    of their own (keyed by seed and k)."""
    V = np.array(V, dtype=np.float64, copy=True)
    th = _rng(seed, 3_000_000 + k).uniform(0.0, 2.0 * np.pi, V.shape[0] - 1)
    c, s = np.cos(th), np.sin(th)
    for j in range(V.shape[0] - 1):
        a, b = V[j].copy(), V[j + 1].copy()
        V[j] = c[j] * a - s[j] * b
        V[j + 1] = s[j] * a + c[j] * b
    return V


def drifting_rows(n: int, d: int, r: int, sigma: np.ndarray, period: int, noise: float = 0.01,
                  seed: int = 0, start: int = 0) -> np.ndarray:
    """Rows start..start+n-1 of a stream whose basis rotates by one Givens
    sweep every `period` rows: row t uses V_k, k = t // period, V_0 = basis(d, r)
    and V_k = G_k V_{k-1}; within a period the rows are those of
    low_rank_noisy with that basis."""
    out = np.empty((n, d), dtype=np.float32)
    V = basis(d, r, seed)
    k_have = 0
    t = start
    while t < start + n:
        k = t // period
        while k_have < k:
            k_have += 1
            V = givens_sweep(V, seed, k_have)
        t1 = min(start + n, (k + 1) * period)
        out[t - start:t1 - start] = low_rank_noisy(t1 - t, d, r, sigma, noise=noise, seed=seed, stream=k,
                                                   start=t - k * period, V=V)
        t = t1
    return out


# The workloads of the persistent setting (d, l, n, rank, spectrum).
WORKLOADS = {
    "small_d256_l32": dict(n=10_000, d=256, ell=32, r=20, spectrum="geometric"),
    "tight_d4096_l1024": dict(n=1_000_000, d=4096, ell=1024, r=200, spectrum="powerlaw"),
}


def workload_rows(name: str, n: int | None = None, start: int = 0, seed: int = 0) -> np.ndarray:
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    return low_rank_noisy(n, w["d"], w["r"], spectrum(w["spectrum"], w["r"]), seed=seed, start=start)


def serving_mix(sessions: int, requests: int, seed: int = 0) -> dict:
    """A serving workload of `sessions` independent streams:
    d = round8(exp U[ln 256, ln 8192]), l uniform on {32, 64, 128, 256, 512}
    clamped to d/2; `requests` batches, each for a uniformly chosen session,
    of b = round(exp U[0, ln 4096]) rows (at least 1)."""
    g = _rng(seed, 2_000_000)
    d = (np.rint(np.exp(g.uniform(np.log(256.0), np.log(8192.0), sessions)) / 8.0) * 8).astype(np.int64)
    ell = np.minimum(g.choice(np.array([32, 64, 128, 256, 512]), sessions), d // 2)
    who = g.integers(0, sessions, requests)
    b = np.maximum(1, np.rint(np.exp(g.uniform(0.0, np.log(4096.0), requests)))).astype(np.int64)
    return {"d": d, "ell": ell, "session": who, "rows": b}
