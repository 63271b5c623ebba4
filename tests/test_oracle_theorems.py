"""Statistical pins of the oracle against the paper's guarantees.

* Theorem 2 (the simultaneous-iteration guarantees quoted from Musco and
  Musco): with eps_SI = 0.4 and q = ceil(ln d / eps_SI), parts 1-3 hold with
  probability at least 99/100.  Checked over 200 seeded draws, and shown to
  fail when the iteration is removed (q = 0), so the checks can catch a
  broken iteration.
* Lemma 1 (the residual bound used by the sliding-window analysis): the
  buffer after a row satisfies ||C^T C||_2 <= 4 theta with probability at
  least (99/100)(1 - (2/(pi sqrt e))/sqrt(d log2 d)).  Checked after every
  row of an ATTP stream.
"""
import math

import numpy as np

from oracle import bounds, philox
from oracle.aerosketch import AeroSketch, default_q, simul_iter
from synth import low_rank_noisy, spectrum


def _si_failures(q: int, trials: int = 200, d: int = 64, m: int = 16, k: int = 4, eps: float = 0.4):
    """Failures of Theorem 2 parts 1, 2, 3 over `trials` draws of A (d x m,
    singular values 0.8^i, random singular vectors) and of Pi (Philox)."""
    fails = np.zeros(3, dtype=int)
    rng = np.random.default_rng(11)
    sig = 0.8 ** np.arange(m)
    for t in range(trials):
        U, _ = np.linalg.qr(rng.standard_normal((d, m)))
        V, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = (U * sig) @ V.T
        Pi = philox.gaussians(11, t, philox.PURPOSE_SI_TEST, t, 1, m * k).reshape(m, k)
        Z, s2 = simul_iter(A, q, Pi)
        Zk = Z[:, :k]
        R = A - Zk @ (Zk.T @ A)
        tail_f = math.sqrt(float(np.sum(sig[k:] ** 2)))   # ||A - A_k||_F
        tail_2 = sig[k]                                     # ||A - A_k||_2
        if np.linalg.norm(R, "fro") > (1 + eps) * tail_f:
            fails[0] += 1
        if np.linalg.norm(R, 2) > (1 + eps) * tail_2:
            fails[1] += 1
        # part 3: u_i^T A A^T u_i = sigma_i^2 and z_i^T A A^T z_i = the Ritz values
        if np.any(np.abs(sig[:k] ** 2 - s2[:k]) > eps * sig[k] ** 2):
            fails[2] += 1
    return fails


def test_theorem2_parts_1_to_3_hold_with_probability_99_percent():
    trials = 200
    q = default_q(64, 0.4)
    fails = _si_failures(q, trials)
    slack = 0.01 + 4 * math.sqrt(0.01 * 0.99 / trials)   # 4 binomial standard deviations over 1/100
    assert np.all(fails / trials <= slack), fails


def test_theorem2_checks_detect_a_missing_iteration():
    # without the q products the basis is a random subspace: part 3 fails far
    # more often than 1/100, so the checks above would notice a broken loop
    fails = _si_failures(0, 200)
    assert fails[2] / 200 > 0.2, fails


def test_lemma1_residual_bound_after_every_row():
    d, ell, n = 48, 6, 600
    A = low_rank_noisy(n, d, 8, spectrum("geometric", 8), noise=0.05, seed=21).astype(np.float64)
    s = AeroSketch(d, ell, seed=21)
    over = 0
    worst = 0.0
    for a in A:
        s.update(a)
        top = float(np.linalg.norm(s.C, 2) ** 2)
        worst = max(worst, top / s.theta)
        if top > 4.0 * s.theta:
            over += 1
    fail_bound = 1.0 - 0.99 * (1.0 - bounds.pi_failure_bound(d))
    assert s.S, "the stream must exercise dumps"
    # per-row events are correlated, so the allowance is the per-event bound
    # with a factor-2 margin rather than a binomial interval
    assert over / n <= 2 * fail_bound, (over, worst)
