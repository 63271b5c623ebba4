"""Brute-force pin of the AeroSketch oracle's control flow on axis-aligned streams.

When every row lies on a coordinate axis, C^T C stays diagonal and Algorithms
4, 5 and 8 reduce to bookkeeping of per-axis energies:
  insert adds ||a||^2 to its axis; a full buffer subtracts lambda_l (the l-th
  largest of the 2l squared singular values, i.e. of the axis energies padded
  with zeros) from every axis and leaves l-1 rows; the power iteration returns
  the largest energy; simultaneous iteration returns the top-k energies; a dump
  moves the axes with energy >= theta into snapshots.
Axis scales 1, 1e2, 1e4, 1e6 keep distinct energy levels apart so that the
iterations converge to working precision; streams whose levels come closer than
a factor of 10, or whose decisions fall within 1% of a threshold, are skipped
(and the test requires most streams to be checkable).
"""
import math

import numpy as np

from oracle.aerosketch import AeroSketch

SCALES = [1.0, 1e2, 1e4, 1e6]


def _model(rows_axis, rows_val, d, ell, eps):
    e = np.zeros(d)
    dumped = np.zeros(d)
    r, F = 0, 0.0
    events, shrinks, ok = [], [], True

    def separated(v):
        nz = np.sort(v[v > 0])[::-1]
        return all(nz[t] >= 10 * nz[t + 1] or nz[t] == nz[t + 1] for t in range(len(nz) - 1))

    def far(x, thr):
        return abs(x - thr) > 0.01 * thr

    for i, (ax, val) in enumerate(zip(rows_axis, rows_val), start=1):
        F += val * val
        theta = eps * F
        e[ax] += val * val
        r += 1
        if r == 2 * ell:
            lam = np.sort(np.concatenate([e[e > 0], np.zeros(2 * ell)]))[::-1][: 2 * ell]
            e = np.maximum(e - lam[ell - 1], 0.0)
            r = ell - 1
            shrinks.append(i)
        ok &= separated(e)
        top = e.max()
        ok &= far(top, theta / 2)
        if not (top >= theta / 2 and top > 0):
            continue
        srt = np.sort(e)[::-1]
        jmax = int(math.ceil(math.log2(min(ell, d))))
        jstop, xi = 0, 0
        for j in range(1, jmax + 1):
            k = min(2 ** j, ell, d)
            ritz = srt[:k]
            ok &= all(far(x, theta) for x in ritz if x > 0)
            if ritz[k - 1] < theta:
                jstop = j
                sel = (e >= theta) & (e > 0)
                xi = int(sel.sum())
                dumped[sel] += e[sel]
                e[sel] = 0.0
                break
        events.append((i, jstop, xi))
    return dict(events=events, shrinks=shrinks, B=np.diag(e + dumped), ok=ok)


def test_bookkeeping_matches_oracle():
    d, ell, eps = 6, 2, 0.3
    checked = 0
    for seed in range(60):
        rng = np.random.default_rng(seed)
        n = 40
        axis = rng.integers(0, 4, size=n)
        val = np.sqrt(np.array([SCALES[a] for a in axis]) * rng.uniform(1.0, 1.5, size=n))
        m = _model(axis, val, d, ell, eps)
        if not m["ok"]:
            continue
        A = np.zeros((n, d))
        A[np.arange(n), axis] = val
        s = AeroSketch(d, ell, eps=eps, seed=seed).run(A)
        got = [(ev.i, ev.j_stop, ev.xi) for ev in s.events]
        assert got == m["events"], seed
        assert s.shrink_rows == m["shrinks"], seed
        B = s.pre_query()
        assert np.abs(B - m["B"]).max() <= 1e-9 * np.trace(m["B"]), seed
        checked += 1
    assert checked >= 20
