"""ATTP historical queries (Algorithm 8 Query(t) = Algorithm 5 with lb = 0,
ub = t) on the GPU against the FP64 oracle, which replays the GPU's decisions
at ties.  For t < T the residual C_t is not stored: B_t is the sum of the
snapshot terms taken at rows <= t.

Bars: B_t entrywise within 1e-5 of trace(A_t^T A_t) (FP32 snapshots), the
covariance error of the historical sketch within 1e-6 of the oracle's."""
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


@pytest.mark.parametrize("d,ell,n,seed,prec", [(32, 6, 400, 3, 0), (64, 8, 900, 4, 0), (64, 8, 900, 4, 3)])
def test_historical_query_parity(d, ell, n, seed, prec):
    p = _gpu()
    A = low_rank_noisy(n, d, 8, spectrum("powerlaw", 8), noise=0.05, seed=seed)
    s = p.Sketch(d, ell, seed=seed, trace=True, prec=prec)
    s.update(A)
    assert s.stats()["device_status"] == 0
    rep = p.binding.replay_from_trace(s.trace())
    A64 = A.astype(np.float64)
    o = AeroSketch(d, ell, seed=seed, replay=rep, tie_rel=1e-5).run(A64)
    assert not o.mismatches, o.mismatches[:5]
    times = sorted({sn.t for sn in o.S})
    assert len(times) >= 4
    checks = sorted({0, 1, times[1], times[1] - 1, times[len(times) // 2], times[-1], n - 1})
    for t in checks:
        At = A64[:t]
        AtA = At.T @ At
        Bg = s.query_gram(t)
        Bo = o.pre_query(ub=t)
        tr = max(np.trace(AtA), 1e-300)
        assert np.abs(Bg - Bo).max() <= 1e-5 * tr, t
        if t == 0:
            assert np.all(Bg == 0.0)
            continue
        eg = cov_err(At, s.query(t), AtA)
        eo = cov_err(At, o.query(ub=t), AtA)
        assert abs(eg - eo) <= 1e-6, (t, eg, eo)
    # t = T is the current-time query (residual included)
    assert np.array_equal(s.query_gram(n), s.query_gram())


def test_historical_query_rejects_bad_times():
    p = _gpu()
    A = low_rank_noisy(50, 16, 4, spectrum("powerlaw", 4), seed=1)
    s = p.Sketch(16, 4)
    s.update(A)
    for t in (-2, 51, 10**9):
        with pytest.raises(p.binding.AeroSketchError):
            s.query(t)
        with pytest.raises(p.binding.AeroSketchError):
            s.query_gram(t)
