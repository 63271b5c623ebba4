"""Closed-form pins of the parity unit (Section 5.1.2's covariance error) and of
the classic Frequent Directions bound.

Every value below is worked out by hand from the definitions, independently of
the code under test:
  cov_err(A, B) = ||A^T A - B^T B||_2 / ||A||_F^2, the spectral norm of the
  symmetric difference being its largest ABSOLUTE eigenvalue;
  fd_bound(A, l) = min over k = 0 .. l-1 of ||A - A_k||_F^2 / (l - k), over
  ||A||_F^2 (A_k the best rank-k approximation, so ||A - A_k||_F^2 is the sum of
  the squared singular values past the k-th).
The cases are chosen so that each plausible slip gives a different number: a
halved result, normalising by ||A||_F instead of ||A||_F^2, max(lambda) instead
of max |lambda|, A A^T or B B^T in place of A^T A or B^T B, and a k range shifted
by one at either end.
"""
import numpy as np
import pytest

from oracle.metric import cov_err, fd_bound


def _diag_rows(sig, n=None):
    """A = [diag(sig); 0] with n >= len(sig) rows."""
    d = len(sig)
    n = n or d
    A = np.zeros((n, d))
    A[np.arange(d), np.arange(d)] = sig
    return A


def test_cov_err_empty_sketch_is_top_energy_share():
    # A^T A = diag(9, 4, 1), B = 0: err = 9 / 14
    A = _diag_rows([3.0, 2.0, 1.0], n=5)
    B = np.zeros((2, 3))
    assert cov_err(A, B) == pytest.approx(9.0 / 14.0, rel=1e-14)


def test_cov_err_top_k_rows_leaves_next_direction():
    # B = the top 2 rows of diag(4, 3, 2, 1): A^T A - B^T B = diag(0, 0, 4, 1),
    # err = sigma_3^2 / sum sigma^2 = 4 / 30
    A = _diag_rows([4.0, 3.0, 2.0, 1.0])
    B = A[:2].copy()
    assert cov_err(A, B) == pytest.approx(4.0 / 30.0, rel=1e-14)


def test_cov_err_takes_the_largest_absolute_eigenvalue():
    # A^T A = diag(4, 1), B^T B = diag(7, 0): the difference diag(-3, 1) has
    # max lambda = 1 but max |lambda| = 3, so err = 3 / 5 (not 1 / 5, not 3 / sqrt 5)
    A = _diag_rows([2.0, 1.0])
    B = np.array([[np.sqrt(7.0), 0.0]])
    assert cov_err(A, B) == pytest.approx(3.0 / 5.0, rel=1e-14)


def test_cov_err_negative_definite_difference():
    # B = 2 A: A^T A - B^T B = -3 A^T A, err = 3 sigma_1^2 / ||A||_F^2 = 3 * 25 / 34
    A = _diag_rows([5.0, 3.0])
    assert cov_err(A, 2.0 * A) == pytest.approx(3.0 * 25.0 / 34.0, rel=1e-14)


def test_cov_err_rotated_square_sketch_distinguishes_transposes():
    # A = U diag(s) V^T (6 x 4), B = diag(t) V^T (4 x 4):
    # A^T A - B^T B = V diag(s^2 - t^2) V^T, err = max |s^2 - t^2| / sum s^2.
    # B B^T = diag(t^2) differs from B^T B, and A A^T is 6 x 6, so a transposed
    # operand gives another number or fails.
    rng = np.random.default_rng(0)
    U, _ = np.linalg.qr(rng.standard_normal((6, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    s = np.array([3.0, 2.0, 1.5, 0.5])
    t = np.array([2.5, 2.0, 0.5, 0.0])
    A = U @ np.diag(s) @ V.T
    B = np.diag(t) @ V.T
    want = np.max(np.abs(s**2 - t**2)) / np.sum(s**2)   # s^2 - t^2 = (2.75, 0, 2, 0.25)
    assert want == pytest.approx(2.75 / 15.5)
    assert cov_err(A, B) == pytest.approx(want, rel=1e-12)


def test_cov_err_given_gram_matches_and_exact_sketch_is_zero():
    A = _diag_rows([3.0, 2.0, 1.0], n=4)
    AtA = A.T @ A
    B = np.zeros((1, 3))
    assert cov_err(A, B, AtA) == pytest.approx(9.0 / 14.0, rel=1e-14)
    assert cov_err(A, A) == 0.0


def test_fd_bound_minimum_at_last_k():
    # sigma^2 = (16, 9, 4, 1), ||A||_F^2 = 30, l = 3:
    #   k = 0: 30 / 3 = 10;  k = 1: 14 / 2 = 7;  k = 2: 5 / 1 = 5  -> 5 / 30
    A = _diag_rows([4.0, 3.0, 2.0, 1.0])
    assert fd_bound(A, 3) == pytest.approx(5.0 / 30.0, rel=1e-14)


def test_fd_bound_minimum_at_k_zero():
    # flat spectrum sigma^2 = (1, 1, 1, 1), l = 3:
    #   k = 0: 4 / 3;  k = 1: 3 / 2;  k = 2: 2 / 1  -> (4/3) / 4 = 1/3
    A = _diag_rows([1.0, 1.0, 1.0, 1.0], n=6)
    assert fd_bound(A, 3) == pytest.approx(1.0 / 3.0, rel=1e-14)


def test_fd_bound_interior_minimum_and_l_one():
    # sigma^2 = (100, 1, 1, 1, 1), total 104, l = 4:
    #   k = 0: 104/4 = 26; k = 1: 4/3; k = 2: 3/2; k = 3: 2/1  -> (4/3) / 104
    A = _diag_rows([10.0, 1.0, 1.0, 1.0, 1.0])
    assert fd_bound(A, 4) == pytest.approx((4.0 / 3.0) / 104.0, rel=1e-14)
    # l = 1 has only k = 0: ||A||_F^2 / 1, normalised to 1
    assert fd_bound(A, 1) == pytest.approx(1.0, rel=1e-14)


def test_cov_err_square_nonsymmetric_stream():
    # A = [[1, 2], [0, 1]]: A^T A = [[1, 2], [2, 5]] but A A^T = [[5, 2], [2, 1]].
    # B = [[1, 0]]: A^T A - B^T B = [[0, 2], [2, 5]], eigenvalues (5 +- sqrt 41) / 2,
    # ||A||_F^2 = 6, so err = (5 + sqrt 41) / 12 (A A^T would give 5 / 6)
    A = np.array([[1.0, 2.0], [0.0, 1.0]])
    B = np.array([[1.0, 0.0]])
    assert cov_err(A, B) == pytest.approx((5.0 + np.sqrt(41.0)) / 12.0, rel=1e-14)
