"""Covariance-error metric, FP64 (oracle; test infrastructure only).

Section 5.1.2 (Metrics): the empirical relative covariance error
||A^T A - B^T B||_2 / ||A||_F^2, with the spectral norm of the symmetric d x d
difference taken as its largest absolute eigenvalue.
"""
from __future__ import annotations

import numpy as np


def gram(A: np.ndarray) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    return A.T @ A


def cov_err(A: np.ndarray, B: np.ndarray, AtA: np.ndarray | None = None) -> float:
    """||A^T A - B^T B||_2 / ||A||_F^2 in FP64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if AtA is None:
        AtA = A.T @ A
    fro2 = float(np.trace(AtA))
    diff = AtA - B.T @ B
    diff = 0.5 * (diff + diff.T)
    return float(np.max(np.abs(np.linalg.eigvalsh(diff)))) / fro2


def fd_bound(A: np.ndarray, ell: int) -> float:
    """min over k < l of ||A - A_k||_F^2 / (l - k), normalised by ||A||_F^2
    (the classic Frequent Directions guarantee)."""
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    s2 = s * s
    fro2 = float(s2.sum())
    tails = fro2 - np.concatenate([[0.0], np.cumsum(s2)])
    best = min(tails[k] / (ell - k) for k in range(ell))
    return best / fro2
