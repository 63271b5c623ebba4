"""The FP64 core eigensolver (through the C ABI) against LAPACK (numpy.linalg.eigh)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    return p


def _check(p, A, nev):
    lam, V = p.binding.symeig(A, nev)
    ref = np.linalg.eigvalsh(A)[::-1][:nev]
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.abs(lam - ref).max() <= 1e-11 * scale * max(1, A.shape[0] / 64)
    # residual and orthogonality of the returned pairs
    R = A @ V - V * lam[None, :]
    assert np.abs(R).max() <= 1e-9 * scale
    assert np.abs(V.T @ V - np.eye(nev)).max() <= 1e-8


@pytest.mark.parametrize("n", [2, 3, 7, 64, 200, 257, 600])
def test_random_spd(n):
    p = _p()
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n + 3))
    _check(p, B @ B.T, max(1, n // 2))


def test_clustered_and_rank_deficient():
    p = _p()
    rng = np.random.default_rng(1)
    n = 300
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([[5.0, 4.0, 4.0 + 1e-12, 3.0], np.full(20, 1.0), np.zeros(n - 24)])
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    lam_g, V = p.binding.symeig(A, 24)
    assert np.abs(lam_g - np.sort(lam)[::-1][:24]).max() <= 1e-11 * 5 * n / 64
    # the invariant subspaces are recovered even where eigenvalues coincide
    P = V @ V.T
    P_ref = Q[:, :24] @ Q[:, :24].T
    assert np.abs(P - P_ref).max() <= 1e-8
    assert np.abs(V.T @ V - np.eye(24)).max() <= 1e-8


def test_zero_and_diagonal():
    p = _p()
    lam, V = p.binding.symeig(np.zeros((40, 40)), 5)
    assert np.all(lam == 0)
    D = np.diag(np.arange(1.0, 301.0))
    lam, V = p.binding.symeig(D, 10)
    assert np.allclose(lam, np.arange(300.0, 290.0, -1), rtol=0, atol=1e-10)


@pytest.mark.parametrize("n,nev", [(2048, 1024), (1024, 512)])
def test_fd_buffer_spectrum(n, nev):
    """The shape of the FD shrink's Gram: a low-rank block of large eigenvalues
    over a wide noise floor (2l = n buffer rows of a rank-200 power-law stream)."""
    p = _p()
    rng = np.random.default_rng(n)
    d, r = 2 * n, 200
    V, _ = np.linalg.qr(rng.standard_normal((d, r)))
    C = (rng.standard_normal((n, r)) / np.arange(1, r + 1)) @ V.T + 0.01 * rng.standard_normal((n, d))
    G = C @ C.T
    _check(p, G, nev)
