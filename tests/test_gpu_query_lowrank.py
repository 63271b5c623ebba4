"""The low-rank route of the query (Algorithm 5 through the stacked factors
F = [C; Z_j^T; Y_j], B = F^T H F) against the FP64 oracle's query and against
the dense d x d route of the same GPU sketch.

Both routes compute the same l x d sketch B_hat up to rounding and the signs of
its rows, so B_hat^T B_hat is compared element by element, within 1e-6 of
||A||_F^2 in Frobenius norm (which bounds the spectral norm, so the two
covariance errors differ by at most 1e-6).  Against the oracle, the covariance
error agrees within 1e-6 (decisions replayed at ties)."""
import numpy as np
import pytest

from oracle.aerosketch import AeroSketch
from oracle.metric import cov_err
from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    return p


def _two_routes(p, A, d, ell, prec, seed):
    lo = p.Sketch(d, ell, seed=seed, trace=True, prec=prec)
    de = p.Sketch(d, ell, seed=seed, prec=prec, dense_query=True)
    lo.update(A)
    de.update(A)
    return lo, de


def _gram_gap(B1, B2):
    B1 = B1.astype(np.float64)
    B2 = B2.astype(np.float64)
    return np.linalg.norm(B1.T @ B1 - B2.T @ B2)


@pytest.mark.parametrize("d,ell,n,r,prec", [(256, 16, 60, 8, 0), (1024, 64, 200, 20, 0), (4096, 256, 700, 40, 3)])
def test_lowrank_query_matches_oracle_and_dense_route(d, ell, n, r, prec):
    p = _gpu()
    A = low_rank_noisy(n, d, r, spectrum("geometric", r), noise=0.01, seed=5)
    lo, de = _two_routes(p, A, d, ell, prec, seed=5)
    st = lo.stats()
    rF = st["rows_in_buffer"] + 2 * st["snapshot_rank"]
    assert 4 * rF <= 3 * d, rF        # the low-rank route applies
    assert st["dumps"] >= 1
    A64 = A.astype(np.float64)
    AtA = A64.T @ A64
    fro2 = float(np.trace(AtA))
    Bl, Bd = lo.query(), de.query()
    assert _gram_gap(Bl, Bd) <= 1e-6 * fro2
    # both routes start from the same B_T
    assert np.array_equal(lo.query_gram(), de.query_gram())
    o = AeroSketch(d, ell, seed=5, replay=p.binding.replay_from_trace(lo.trace()), tie_rel=1e-5).run(A64)
    assert not o.mismatches, o.mismatches[:3]
    eg, eo = cov_err(A, Bl, AtA), cov_err(A, o.query(), AtA)
    assert abs(eg - eo) <= 1e-6, (eg, eo)
    assert eg <= 2.0 / ell


def test_lowrank_query_d8192_matches_dense_route():
    """d = 8192, l = 512 (the largest C4 session): the r_F x r_F route against
    the 8192 x 8192 one."""
    p = _gpu()
    d, ell, n = 8192, 512, 1200
    A = low_rank_noisy(n, d, 20, spectrum("geometric", 20), noise=0.01, seed=6)
    lo, de = _two_routes(p, A, d, ell, 3, seed=6)
    st = lo.stats()
    rF = st["rows_in_buffer"] + 2 * st["snapshot_rank"]
    assert 4 * rF <= 3 * d and st["dumps"] >= 1
    fro2 = float(np.sum(A.astype(np.float64) ** 2))
    assert _gram_gap(lo.query(), de.query()) <= 1e-6 * fro2


def test_lowrank_historical_query_and_empty_sketch():
    p = _gpu()
    d, ell = 512, 32
    A = low_rank_noisy(200, d, 10, spectrum("geometric", 10), noise=0.01, seed=7)
    lo, de = _two_routes(p, A, d, ell, 0, seed=7)
    fro2 = float(np.sum(A.astype(np.float64) ** 2))
    for t in (1, 57, 150, 199):        # historical: snapshot terms with t_j <= t only
        assert _gram_gap(lo.query(t), de.query(t)) <= 1e-6 * fro2
    e = p.Sketch(d, ell)
    assert np.all(e.query() == 0)
