"""Exact Frequent Directions, FP64 (oracle; test infrastructure only).

Frequent Directions (Section 2.3, the FD paragraph and its two displayed
equations): a 2l x d buffer; a row goes into an empty row; when all 2l rows
are full, SVD the buffer, subtract sigma_l^2 from every squared singular value
(clamped at zero) and keep Sigma' V^T, which leaves rows l..2l empty.

Rows are kept in the canonical order used across the oracle: after a shrink
the retained rows are the singular directions in descending order at indices
0..l-2, and the next row is inserted at index l-1.
"""
from __future__ import annotations

import numpy as np


class ExactFD:
    def __init__(self, d: int, ell: int):
        if not (1 <= ell and 2 * ell <= d):
            raise ValueError("Frequent Directions needs 1 <= l <= d/2")
        self.d, self.ell = d, ell
        self.B = np.zeros((2 * ell, d), dtype=np.float64)
        self.r = 0
        self.shrinks = 0
        self.delta_sum = np.zeros((d, d), dtype=np.float64)  # sum of shrink losses

    def update(self, a: np.ndarray) -> None:
        self.B[self.r] = a
        self.r += 1
        if self.r == 2 * self.ell:
            _, s, vt = np.linalg.svd(self.B, full_matrices=False)
            s2 = s * s
            s2_ell = s2[self.ell - 1]
            kept = np.sqrt(np.maximum(s2 - s2_ell, 0.0))
            loss = np.minimum(s2, s2_ell)
            self.delta_sum += (vt.T * loss) @ vt
            self.B = kept[:, None] * vt
            self.B[self.ell - 1:] = 0.0
            self.r = self.ell - 1
            self.shrinks += 1

    def run(self, A: np.ndarray) -> "ExactFD":
        for a in np.asarray(A, dtype=np.float64):
            self.update(a)
        return self

    def sketch(self) -> np.ndarray:
        return self.B[: self.r].copy()
