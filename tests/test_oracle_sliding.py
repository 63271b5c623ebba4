"""Pins of the sliding-window oracle (Algorithm 6 with readings R15, R16).

* Exact window: when every row is heavy at level 0 (||a||^2 >= eps N) and the
  window fits the queue cap, level 0 holds exactly the last N rows as raw
  rows, so B = A_w^T A_w of the window (T-N, T] exactly: an off-by-one in the
  expiry test or the query range fails.
* Queue invariants after every row: len <= 8/eps + 1, every item has
  t > T - N (expired items were popped at the row's start), times increase,
  and s follows R15 (previous t + 1, or 1 after an empty queue).
* The query of a drifting stream stays within 2 eps of the window's mass.
"""
import numpy as np
import pytest

from oracle.metric import cov_err
from oracle.sliding import SlidingAeroSketch, levels_for
from synth import low_rank_noisy, spectrum


def test_levels_cover_fact1():
    assert levels_for(1.0) == 1 and levels_for(2.0) == 2 and levels_for(1000.0) == 11


@pytest.mark.parametrize("N,n", [(20, 90), (32, 70)])
def test_all_raw_window_is_exact(N, n):
    d, ell = 24, 8                      # eps = 1/4, cap = 32 >= N
    A = low_rank_noisy(n, d, 6, spectrum("geometric", 6), seed=3)
    A = A.astype(np.float64)
    A *= np.sqrt(1.5 * (2.0 / ell) * N) / np.sqrt(np.min(np.sum(A * A, axis=1)))   # ||a||^2 >= 1.5 eps N
    s = SlidingAeroSketch(d, ell, N, R=float(np.max(np.sum(A * A, axis=1))))
    for T in range(1, n + 1):
        s.update(A[T - 1])
        if T % 7 == 0 or T == n:
            assert s.level_for_query() == 0
            W = A[max(0, T - N):T]
            assert np.abs(s.pre_query() - W.T @ W).max() <= 1e-12 * np.sum(W * W)


def test_queue_invariants():
    d, ell, N = 32, 4, 40
    A = low_rank_noisy(400, d, 6, spectrum("powerlaw", 6), noise=0.05, seed=5).astype(np.float64)
    A *= 3.0
    s = SlidingAeroSketch(d, ell, N, R=float(np.max(np.sum(A * A, axis=1))))
    for a in A:
        s.update(a)
        for Q in s.S:
            assert len(Q) <= s.cap + 1
            prev = None
            for k, it in enumerate(Q):
                assert it.t > s.T - N
                if prev is not None:
                    assert it.t > prev.t and it.s == prev.t + 1
                prev = it
    assert sum(len(Q) for Q in s.S) > 0


@pytest.mark.parametrize("seed", [1, 2])
def test_window_query_error(seed):
    d, ell, N = 32, 8, 120
    A1 = low_rank_noisy(300, d, 6, spectrum("geometric", 6), noise=0.05, seed=seed, stream=1)
    A2 = low_rank_noisy(300, d, 6, spectrum("geometric", 6), noise=0.05, seed=seed + 10, stream=2)
    A = np.vstack([A1, 2.0 * A2]).astype(np.float64)       # the window's mass changes under the stream
    s = SlidingAeroSketch(d, ell, N, R=float(np.max(np.sum(A * A, axis=1))))
    for T in range(1, len(A) + 1):
        s.update(A[T - 1])
        if T % 60 == 0:
            W = A[max(0, T - N):T]
            assert cov_err(W, s.query()) <= 2.0 * s.eps, T
