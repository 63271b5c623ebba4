"""Sliding-window ML-AeroSketch (Algorithm 6) on the GPU against the FP64
oracle, which replays each level's decisions at ties.

* Exact window: every row heavy at level 0 and the window within the queue
  cap: the window's B is the Gram of exactly the last N rows (FP32 products
  summed in FP64 chunks: 1e-6 of its trace; one row too many or too few moves
  it by about 5%).
* Parity on a stream whose window mass changes: at every query time the same
  level answers; B within 1e-5 of trace(A_w^T A_w); covariance error within
  1e-6; queue counters equal."""
import numpy as np
import pytest

from oracle.metric import cov_err
from oracle.sliding import SlidingAeroSketch
from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    return p


def test_all_raw_window_is_exact():
    p = _gpu()
    d, ell, N, n = 24, 8, 20, 90
    A = low_rank_noisy(n, d, 6, spectrum("geometric", 6), seed=3).astype(np.float64)
    A *= np.sqrt(1.5 * (2.0 / ell) * N) / np.sqrt(np.min(np.sum(A * A, axis=1)))
    A = A.astype(np.float32)
    R = float(np.max(np.sum(A.astype(np.float64) ** 2, axis=1)))
    w = p.SlidingWindow(d, ell, N, R)
    for t0 in range(0, n, 13):
        w.update(A[t0:t0 + 13])
        T = min(n, t0 + 13)
        B, lvl = w.query_gram()
        assert lvl == 0
        W = A[max(0, T - N):T].astype(np.float64)
        assert np.abs(B - W.T @ W).max() <= 1e-6 * np.sum(W * W)


@pytest.mark.parametrize("d,ell,N,blk,seed,prec", [(32, 8, 120, 37, 1, 0), (48, 6, 200, 50, 2, 0),
                                                  (256, 128, 400, 97, 3, 3)])
def test_sliding_parity(d, ell, N, blk, seed, prec):
    """prec 3 (split-BF16 x6) with 2l = 256: each level's batched iterations run
    on tcgen05 once its buffer passes 128 rows, and its Gram rows and FD
    rebuilds on the tcgen05 GEMM."""
    p = _gpu()
    A1 = low_rank_noisy(300, d, 6, spectrum("geometric", 6), noise=0.05, seed=seed, stream=1)
    A2 = low_rank_noisy(300, d, 6, spectrum("geometric", 6), noise=0.05, seed=seed + 10, stream=2)
    A = np.vstack([A1, 2.0 * A2]).astype(np.float32)
    A64 = A.astype(np.float64)
    R = float(np.max(np.sum(A64 * A64, axis=1)))
    w = p.SlidingWindow(d, ell, N, R, seed=seed, trace=True, prec=prec)
    got = {}
    for t0 in range(0, len(A), blk):
        w.update(A[t0:t0 + blk])
        T = min(len(A), t0 + blk)
        B, lvl = w.query_gram()
        Bh, lvl2 = w.query()
        got[T] = (B, lvl, Bh)
    st = w.stats()
    L = st["levels"]
    rep = [p.binding.replay_from_trace(w.level(j).trace()) for j in range(L)]
    o = SlidingAeroSketch(d, ell, N, R, seed=seed, replay=rep, tie_rel=1e-5)
    assert o.L == L
    for T in range(1, len(A) + 1):
        o.update(A64[T - 1])
        if T in got:
            B, lvl, Bh = got[T]
            assert lvl == o.level_for_query(), T
            W = A64[max(0, T - N):T]
            WtW = W.T @ W
            assert np.abs(B - o.pre_query()).max() <= 1e-5 * np.trace(WtW), T
            assert abs(cov_err(W, Bh, WtW) - cov_err(W, o.query(), WtW)) <= 1e-6, T
    for lv in o.levels:
        assert not lv.mismatches, lv.mismatches[:5]
    assert st["raw_queued"] == sum(1 for Q in o.S for it in Q if it.a is not None)
    assert st["snapshots_queued"] == sum(1 for Q in o.S for it in Q if it.a is None)


def test_sliding_rejects_bad_arguments():
    p = _gpu()
    with pytest.raises(p.AeroSketchError):
        p.SlidingWindow(16, 2, 0, 4.0)
    with pytest.raises(p.AeroSketchError):
        p.SlidingWindow(16, 2, 10, 0.5)
    w = p.SlidingWindow(16, 2, 10, 4.0)
    bad = np.zeros((3, 16), dtype=np.float32)
    bad[1, 2] = np.nan
    with pytest.raises(p.AeroSketchError):
        w.update(bad)
