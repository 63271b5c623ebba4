"""Pins of the P5 oracle (Algorithm 10 with readings R13, R14).

* Exact bookkeeping: a dump moves its snapshot term from C'^T C' to the
  coordinator exactly and an FD shrink drops a PSD Delta, so
  A^T A = B + sum_j C_j^T C_j + sum_j sum_i Delta_{j,i} up to rounding.
* Message conservation: F_hat plus the sites' unsent F_j is ||A||_F^2, every
  unsent F_j lies below the site's trigger, one broadcast per m messages.
* Before the first broadcast theta = inf (R13): the sites run exact FD and
  send nothing; the broadcast after m messages sets theta = (eps/m) F_hat.
* The final query meets a loose error bound (2 eps ||A||_F^2).
"""
import numpy as np
import pytest

from oracle.metric import cov_err
from oracle.p5 import P5
from synth import basis, low_rank_noisy, spectrum


def _sites(m, n, d, seed, r=6):
    V = basis(d, r, seed=seed)
    return [low_rank_noisy(n, d, r, spectrum("geometric", r), noise=0.05, seed=seed, stream=j + 1, V=V).astype(np.float64)
            for j in range(m)]


def _run(m, n, d, ell, b, seed, **kw):
    rows = _sites(m, n, d, seed)
    p = P5(d, ell, m, seed=seed, **kw)
    for t0 in range(0, n, b):
        p.round([x[t0:t0 + b] for x in rows])
    return p, rows


@pytest.mark.parametrize("m,n,d,ell,b,seed", [(4, 120, 24, 4, 10, 1), (6, 90, 32, 4, 15, 2)])
def test_p5_exact_bookkeeping(m, n, d, ell, b, seed):
    p, rows = _run(m, n, d, ell, b, seed, track_delta=True)
    A = np.vstack(rows)
    AtA = A.T @ A
    rhs = p.B + p.residual_gram() + sum(s.delta_sum for s in p.sites)
    assert np.abs(AtA - rhs).max() <= 1e-10 * np.trace(AtA)
    lam = np.linalg.eigvalsh(AtA - p.B - p.residual_gram())
    assert lam[0] >= -1e-10 * np.trace(AtA)
    assert p.sent_snapshots > 0 and p.broadcasts > 0


@pytest.mark.parametrize("m,n,b", [(4, 120, 10), (5, 77, 7)])
def test_p5_message_conservation(m, n, b):
    p, rows = _run(m, n, 24, 4, b, 3)
    total = sum(float(np.sum(x * x)) for x in rows)
    assert abs(p.F_hat + sum(p.F) - total) <= 1e-12 * total
    for f in p.F:
        assert f < (p.eps / p.m) * p.F_site or f == 0.0
    assert p.broadcasts >= 1
    for s in p.sites:
        assert s.theta == (p.eps / p.m) * p.F_site


def test_p5_first_round_is_exact_fd_and_sends_nothing():
    from oracle.fd import ExactFD
    m, d, ell = 3, 20, 4
    rows = _sites(m, 12, d, 4)         # 12 rows per site: one FD shrink
    p = P5(d, ell, m)
    p.round(rows)                      # theta = inf until the broadcast at the round's end
    assert p.sent_snapshots == 0 and np.all(p.B == 0.0)
    assert p.broadcasts == 12          # F_hat = 0 before: every row sent its F_j, 36 messages / m
    for j in range(m):
        fd = ExactFD(d, ell)
        for a in rows[j]:
            fd.update(a)
        Cs, Cf = p.sites[j].C, fd.B
        assert np.abs(Cs.T @ Cs - Cf.T @ Cf).max() <= 1e-9 * np.sum(rows[j] ** 2)
    theta = (p.eps / m) * sum(float(np.sum(x * x)) for x in rows)
    assert all(abs(s.theta - theta) <= 1e-12 * theta for s in p.sites)


def test_p5_query_error_bound():
    p, rows = _run(6, 200, 32, 6, 20, 5)
    A = np.vstack(rows)
    assert cov_err(A, p.query()) <= 2.0 * p.eps
