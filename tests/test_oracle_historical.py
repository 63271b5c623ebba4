"""Pins of the oracle's ATTP historical query (Algorithm 8 Query(t) =
Algorithm 5 with lb = 0, ub = t; reading R12: no residual C_t for t < T).

* Time filter: the historical B_t computed at the end of the stream equals
  the current-time B taken at time t minus C_t^T C_t, at every checkpoint,
  including the rows where a snapshot was taken (t_j = t is included, later
  snapshots are not).
* Telescoping (the ATTP error analysis: a dump moves exactly its snapshot
  term out of C'^T C', an FD shrink drops a PSD Delta): A_t^T A_t - C_t^T C_t
  - B_t is positive semidefinite.
"""
import numpy as np
import pytest

from oracle.aerosketch import AeroSketch
from synth import low_rank_noisy, spectrum


def _stream(n, d, seed, kind="geometric"):
    return low_rank_noisy(n, d, 8, spectrum(kind, 8), seed=seed).astype(np.float64)


# fixed theta (Algorithm 3's threshold) gives a snapshot every few rows;
# theta = None runs the ATTP threshold of Algorithm 8
@pytest.mark.parametrize("d,ell,n,seed,theta", [(24, 3, 160, 1, 1500.0), (32, 4, 220, 2, 2500.0),
                                                 (24, 6, 150, 3, None)])
def test_historical_gram_matches_state_at_t(d, ell, n, seed, theta):
    A = _stream(n, d, seed, "geometric" if theta is not None else "powerlaw")
    s = (AeroSketch(d, ell, seed=seed) if theta is None
         else AeroSketch(d, ell, seed=seed, theta_mode="fixed", theta_fixed=theta))
    ref = {}
    for i, a in enumerate(A, start=1):
        s.update(a)
        ref[i] = s.pre_query() - s.C.T @ s.C
    dump_times = sorted({sn.t for sn in s.S})
    assert len(dump_times) >= (5 if theta is not None else 2)
    checks = set(dump_times[:: max(1, len(dump_times) // 6)]) | {t - 1 for t in dump_times[:3]} | {n // 2, n - 1}
    scale = float(np.sum(A * A))
    for t in sorted(c for c in checks if 1 <= c < n):
        H = s.pre_query(ub=t)
        assert np.max(np.abs(H - ref[t])) <= 1e-12 * scale, t
    assert np.all(s.pre_query(ub=0) == 0.0)


@pytest.mark.parametrize("d,ell,n,seed,theta", [(24, 3, 200, 5, 1500.0), (40, 5, 260, 6, 3000.0),
                                                 (24, 6, 200, 7, None)])
def test_historical_gram_telescoping_psd(d, ell, n, seed, theta):
    A = _stream(n, d, seed, "geometric" if theta is not None else "powerlaw")
    s = (AeroSketch(d, ell, seed=seed) if theta is None
         else AeroSketch(d, ell, seed=seed, theta_mode="fixed", theta_fixed=theta))
    resid = {}
    for i, a in enumerate(A, start=1):
        s.update(a)
        if i % 17 == 0:
            resid[i] = s.C.T @ s.C
    for t, CtC in resid.items():
        At = A[:t]
        D = At.T @ At - CtC - s.pre_query(ub=t)
        lam_min = np.linalg.eigvalsh(0.5 * (D + D.T))[0]
        assert lam_min >= -1e-10 * float(np.sum(At * At)), t


def test_historical_query_shrinks_and_validates():
    A = _stream(150, 24, 9)
    s = AeroSketch(24, 3, theta_mode="fixed", theta_fixed=1500.0).run(A)
    t = sorted({sn.t for sn in s.S})[3]
    Bh = s.query(ub=t)
    B = s.pre_query(ub=t)
    lam = np.sort(np.linalg.eigvalsh(B))[::-1]
    # the eigen-shrink of Algorithm 5: B_hat^T B_hat = sum_j max(lam_j - lam_l, 0) v_j v_j^T
    got = np.sort(np.linalg.eigvalsh(Bh.T @ Bh))[::-1][:3]
    want = np.maximum(lam[:3] - lam[2], 0.0)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * lam[0])
    with pytest.raises(ValueError):
        s.pre_query(ub=s.T + 1)
    with pytest.raises(ValueError):
        s.pre_query(ub=-1)
