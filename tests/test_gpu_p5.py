"""P5 (Algorithm 10), merging by decomposability and the site/coordinator
calls, on the GPU through the C ABI.

P5 parity: the GPU runtime and the FP64 oracle run the same synchronous
rounds; the oracle replays each GPU site's decisions at ties.  The message
protocol depends only on row norms, so its counters must match exactly; the
coordinator's B within 1e-5 of trace(A^T A) (FP32 snapshots), the query's
covariance error within 1e-6."""
import numpy as np
import pytest

from oracle.metric import cov_err
from oracle.p5 import P5 as OracleP5
from synth import basis, low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    return p


def _sites(m, n, d, seed, r=6):
    V = basis(d, r, seed=seed)
    return [low_rank_noisy(n, d, r, spectrum("geometric", r), noise=0.05, seed=seed, stream=j + 1, V=V)
            for j in range(m)]


@pytest.mark.parametrize("m,n,d,ell,b,seed,prec", [(4, 120, 32, 4, 10, 1, 0), (3, 200, 64, 8, 25, 2, 0),
                                                  (5, 90, 48, 6, 9, 3, 0), (2, 320, 256, 128, 64, 4, 3)])
def test_p5_parity(m, n, d, ell, b, seed, prec):
    """prec 3 (split-BF16 x6) with 2l = 256: the sites' batched iterations run on
    tcgen05 once a block's buffer passes 128 rows, and their Gram rows and FD
    rebuilds on the tcgen05 GEMM."""
    p = _gpu()
    rows = _sites(m, n, d, seed)
    g = p.P5(d, ell, m, seed=seed, trace=True, prec=prec)
    for t0 in range(0, n, b):
        g.round([x[t0:t0 + b] for x in rows])
    rep = [p.binding.replay_from_trace(g.site(j).trace()) for j in range(m)]
    o = OracleP5(d, ell, m, seed=seed, replay=rep, tie_rel=1e-5)
    for t0 in range(0, n, b):
        o.round([x[t0:t0 + b].astype(np.float64) for x in rows])
    for s in o.sites:
        assert not s.mismatches, s.mismatches[:5]
    st = g.stats()
    assert st["messages"] == o.messages
    assert st["broadcasts"] == o.broadcasts
    assert st["snapshots_sent"] == o.sent_snapshots
    assert abs(st["f_hat"] - o.F_hat) <= 1e-12 * o.F_hat
    A = np.vstack(rows).astype(np.float64)
    AtA = A.T @ A
    assert np.abs(g.query_gram() - o.B).max() <= 1e-5 * np.trace(AtA)
    eg, eo = cov_err(A, g.query(), AtA), cov_err(A, o.query(), AtA)
    assert abs(eg - eo) <= 1e-6, (eg, eo)
    assert eg <= 2.0 * o.eps


def test_merge_is_decomposable():
    p = _gpu()
    d, ell = 48, 6
    A1 = low_rank_noisy(300, d, 8, spectrum("powerlaw", 8), seed=4, stream=1)
    A2 = low_rank_noisy(250, d, 8, spectrum("powerlaw", 8), seed=4, stream=2)
    s1 = p.Sketch(d, ell, seed=1)
    s2 = p.Sketch(d, ell, seed=2)
    s1.update(A1)
    s2.update(A2)
    g1, g2 = s1.query_gram(), s2.query_gram()
    s1.merge(s2)
    assert np.abs(s1.query_gram() - (g1 + g2)).max() <= 1e-12 * np.trace(g1 + g2)
    assert np.array_equal(s2.query_gram(), g2)          # src is not modified
    A = np.vstack([A1, A2]).astype(np.float64)
    AtA = A.T @ A
    # each part errs by at most 2/l of its own mass (the deterministic bound);
    # the merged Gram errs by at most their sum, and the query shrink adds at
    # most the same again (Weyl, as for a single stream)
    e = cov_err(A, s1.query(), AtA)
    assert e <= 2.0 * 2.0 / ell
    # merging keeps later updates working: s1's own rows stay its own
    s1.update(A1[:10])
    assert s1.stats()["device_status"] == 0


def test_send_snapshots_conserves_the_query_gram():
    p = _gpu()
    d, ell = 32, 4
    A = low_rank_noisy(200, d, 6, spectrum("geometric", 6), seed=5)
    site = p.Sketch(d, ell, mode=p.AS_SITE, theta=500.0, seed=5)
    coord = p.Sketch(d, ell, mode=p.AS_COORDINATOR)
    site.update(A)
    before = site.query_gram()
    dumps = site.stats()["dumps"]
    assert dumps > 0
    n = site.send_snapshots(coord)
    assert n == dumps
    assert np.abs(site.query_gram() + coord.query_gram() - before).max() <= 1e-10 * np.trace(before)
    assert site.send_snapshots(coord) == 0
    assert site.stats()["snapshots_sent"] == n and coord.stats()["snapshots_received"] == n
    site.set_theta(float("inf"))
    site.update(A[:20])
    assert site.send_snapshots(coord) == 0      # theta = inf: exact FD, nothing to send


def test_site_and_coordinator_errors():
    p = _gpu()
    d, ell = 16, 2
    s = p.Sketch(d, ell)                          # persistent: theta is not settable
    with pytest.raises(p.AeroSketchError):
        s.set_theta(1.0)
    f = p.Sketch(d, ell, mode=p.AS_FIXED_THETA, theta=1.0)
    with pytest.raises(p.AeroSketchError):
        f.set_theta(-1.0)
    coord = p.Sketch(d, ell, mode=p.AS_COORDINATOR)
    with pytest.raises(p.AeroSketchError):
        coord.update(np.zeros((3, d), dtype=np.float32))
    other = p.Sketch(2 * d, ell)
    with pytest.raises(p.AeroSketchError):
        coord.merge(other)
    with pytest.raises(p.AeroSketchError):
        other.send_snapshots(coord)
    with pytest.raises(p.AeroSketchError):
        p.Sketch(d, ell, mode=p.binding.AS_SLIDING)
