"""Grouped updates (sketch_update_many) and the serving runtime (as_server)
through the C ABI.

A sketch's kernels and launch shapes depend only on its own configuration and
rows, so every result here is compared BITWISE with the same sketch fed the
same rows alone; admission is checked against sketch_footprint, which must
equal the device bytes a reserved sketch holds.
"""
import numpy as np
import pytest

from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu

SHAPES = [(64, 8), (256, 32), (512, 64), (96, 12), (1024, 160)]


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    return p


def _rows(n, d, seed):
    return low_rank_noisy(n, d, 8, spectrum("powerlaw", 8), noise=0.05, seed=seed)


def _alone(p, d, ell, blocks, seed):
    s = p.Sketch(d, ell, seed=seed, trace=True)
    for b in blocks:
        s.update(b)
    return s


def _same(a, b):
    assert np.array_equal(a.query_gram(), b.query_gram())
    ta = [(e["i"], e["j_stop"], e["xi"], e["sig2_pi"]) for e in a.trace()]
    tb = [(e["i"], e["j_stop"], e["xi"], e["sig2_pi"]) for e in b.trace()]
    assert ta == tb


@pytest.mark.parametrize("d,ell", [(64, 8), (1024, 160)])
def test_footprint_is_the_reserved_device_bytes(d, ell):
    p = _gpu()
    for rank in (0, 37):
        s = p.Sketch(d, ell)
        s.reserve(rank)
        assert s.stats()["device_bytes"] == p.footprint(d, ell, snapshot_rank=rank)


@pytest.mark.parametrize("mode", ["update_many", "update_grouped"])
def test_update_many_is_bitwise_the_sketches_alone(mode):
    p = _gpu()
    upd = getattr(p, mode)
    rng = np.random.default_rng(3)
    sk, blocks, plan = [], [], []
    for t, (d, ell) in enumerate(SHAPES):
        A = _rows(int(rng.integers(150, 400)), d, seed=10 + t)
        sk.append(p.Sketch(d, ell, seed=t, trace=True))
        plan.append((d, ell, A))
    # two rounds; in the second the first sketch appears twice (in list order)
    cut = [len(A) // 2 for _, _, A in plan]
    upd(sk, [A[:c] for (_, _, A), c in zip(plan, cut)])
    upd([sk[0]] + sk, [plan[0][2][cut[0]:cut[0] + 40]] +
                  [A[c + 40:] if t == 0 else A[c:] for t, ((_, _, A), c) in enumerate(zip(plan, cut))])
    for t, (d, ell, A) in enumerate(plan):
        c = cut[t]
        blocks = [A[:c], A[c:c + 40], A[c + 40:]] if t == 0 else [A[:c], A[c:]]
        _same(sk[t], _alone(p, d, ell, blocks, seed=t))
    # grouped: the sketches' batched iterations did share cooperative launches
    grouped = sum(s.stats()["grouped_batches"] for s in sk)
    assert (grouped > 0) if mode == "update_grouped" else (grouped == 0)


def test_server_sessions_are_bitwise_the_sketches_alone():
    p = _gpu()
    rng = np.random.default_rng(4)
    sv = p.Server(workers=8)
    sess, feeds = [], []
    for t, (d, ell) in enumerate(SHAPES):
        sid = sv.open(d, ell, seed=t, trace=True, mass_ratio=1e4)
        sess.append(sid)
        A = _rows(int(rng.integers(200, 500)), d, seed=20 + t)
        cuts = np.sort(rng.choice(np.arange(1, len(A)), size=3, replace=False))
        feeds.append((d, ell, np.split(A, cuts)))
    # all requests queued at once, interleaved across sessions
    order = [(t, k) for k in range(4) for t in range(len(SHAPES))]
    tickets = [(sv.submit(sess[t], feeds[t][2][k]), t, k) for t, k in order]
    lat = [sv.wait(tk) for tk, _, _ in tickets]
    assert all(x > 0.0 for x in lat)
    st = sv.stats()
    assert st["requests_done"] == len(order) and st["requests_failed"] == 0
    assert st["rows_done"] == sum(len(b) for _, _, bl in feeds for b in bl)
    assert 0.0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for t, (d, ell, bl) in enumerate(feeds):
        _same(sv.sketch(sess[t]), _alone(p, d, ell, bl, seed=t))
    sv.close()


def test_admission_by_footprint():
    p = _gpu()
    d, ell, ratio = 512, 64, 100.0
    eps = 2.0 / ell
    rank = int(np.ceil((2.0 / eps) * np.log(2.0 * ratio / eps)))
    fp = p.footprint(d, ell, snapshot_rank=rank)
    sv = p.Server(hbm_budget=fp + fp // 2, workers=2)
    a = sv.open(d, ell, mass_ratio=ratio)
    st = sv.stats()
    assert st["footprint_bytes"] == fp and st["sessions_open"] == 1
    assert sv.sketch(a).stats()["device_bytes"] == fp
    with pytest.raises(p.AeroSketchError) as e:
        sv.open(d, ell, mass_ratio=ratio)
    assert "AS_EBUSY" in str(e.value)
    assert sv.stats()["sessions_refused"] == 1
    sv.close_session(a)
    assert sv.stats()["footprint_bytes"] == 0
    b = sv.open(d, ell, mass_ratio=ratio)          # the freed budget admits it
    sv.wait(sv.submit(b, _rows(100, d, seed=5)))
    sv.close()


def test_server_errors_and_failed_request():
    p = _gpu()
    d, ell = 64, 8
    sv = p.Server(workers=2)
    with pytest.raises(p.AeroSketchError):
        sv.open(d, 40)                               # ell > d/2
    with pytest.raises(p.AeroSketchError):
        sv.open(d, ell, mass_ratio=0.5)              # a mass ratio is >= 1
    with pytest.raises(p.AeroSketchError):
        sv.submit(12345, _rows(10, d, seed=1))       # no such session
    sid = sv.open(d, ell)
    bad = _rows(30, d, seed=2)
    bad[7, 3] = np.nan
    with pytest.raises(p.AeroSketchError) as e:
        sv.wait(sv.submit(sid, bad))
    assert "AS_EINVAL" in str(e.value)
    assert sv.stats()["requests_failed"] == 1
    sv.wait(sv.submit(sid, _rows(50, d, seed=3)))   # the session keeps serving
    assert sv.sketch(sid).stats()["device_status"] == 0
    sv.close()
