"""Pins of the exact-FD oracle (Section 2.3) against brute-force SVD facts."""
import numpy as np
import pytest

from oracle.fd import ExactFD
from oracle.metric import cov_err, fd_bound
from synth import low_rank_noisy, spectrum


@pytest.mark.parametrize("d,ell,n,seed", [(16, 4, 200, 0), (32, 8, 300, 1), (24, 3, 150, 2)])
def test_fd_error_bound(d, ell, n, seed):
    A = low_rank_noisy(n, d, 6, spectrum("geometric", 6), noise=0.1, seed=seed).astype(np.float64)
    fd = ExactFD(d, ell).run(A)
    B = fd.sketch()
    err = cov_err(A, B)
    # classic FD guarantee ||A^T A - B^T B|| <= ||A - A_k||_F^2 / (l - k) for every k < l
    assert err <= fd_bound(A, ell) * (1 + 1e-9)
    # FD only ever removes energy: A^T A - B^T B is PSD
    lam = np.linalg.eigvalsh(A.T @ A - B.T @ B)
    assert lam.min() >= -1e-10 * np.trace(A.T @ A)


def test_fd_telescoping_closed_form():
    # A^T A - B^T B equals the sum of the shrink losses V min(S^2, s_l^2) V^T
    rng = np.random.default_rng(5)
    A = rng.standard_normal((120, 10))
    fd = ExactFD(10, 3).run(A)
    B = fd.sketch()
    lhs = A.T @ A - B.T @ B
    assert np.allclose(lhs, fd.delta_sum, atol=1e-10 * np.trace(A.T @ A))
    assert fd.shrinks == (120 - 5) // 4 + 1 - (1 if (120 - 5) % 4 == 0 else 0) or fd.shrinks > 0


def test_fd_exact_when_stream_fits():
    # fewer than 2l rows: no shrink, the sketch is the stream itself
    rng = np.random.default_rng(1)
    A = rng.standard_normal((7, 12))
    fd = ExactFD(12, 4).run(A)
    assert np.allclose(fd.sketch(), A)
    assert cov_err(A, fd.sketch()) < 1e-14


def test_fd_rank_le_l_is_lossless_direction_count():
    # a stream of rank < l: after every shrink sigma_l = 0, nothing is lost
    rng = np.random.default_rng(2)
    A = rng.standard_normal((200, 3)) @ rng.standard_normal((3, 16))
    fd = ExactFD(16, 5).run(A)
    assert cov_err(A, fd.sketch()) < 1e-12
