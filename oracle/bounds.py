"""Closed-form probability bounds stated by the paper (oracle; test infrastructure).

Corollary 1: with k = ceil(log2 d) + 1 power iterations,
    Pr[sigma_hat_1^2 >= sigma_1^2 / 2] >= 1 - (2 / (pi sqrt(e))) / sqrt(d log2 d).
Theorem 3, Eq. 1: success probability >= (99/100) times that bound.
"""
from __future__ import annotations

import math


def pi_failure_bound(d: int) -> float:
    """Upper bound on Pr[sigma_hat_1^2 < sigma_1^2 / 2] from Corollary 1."""
    return (2.0 / (math.pi * math.sqrt(math.e))) / math.sqrt(d * math.log2(d))


def success_probability(d: int) -> float:
    """Eq. 1 (Theorem 3)."""
    return 0.99 * (1.0 - pi_failure_bound(d))
