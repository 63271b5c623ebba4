"""Probability amplification (Algorithm 7) on the GPU through the C ABI,
against the FP64 oracle.

Each doubling step of a row whose gate passes runs r simultaneous iterations
(eps_SI = 0.2) and keeps the one whose residual has the smallest estimated top
eigenvalue.  Parity: the oracle replays the GPU's gate, stop, xi and kept-SI
decisions only inside the 1e-5 relative tie band (FP32 storage of C moves the
estimates by ~1e-7 relative) and must agree everywhere else; the kept
choices are compared one by one; the covariance errors agree within 1e-6.
"""
import numpy as np
import pytest

from oracle.aerosketch import AeroSketch
from oracle.metric import cov_err
from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu

TIE = 1e-5


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    return p


def _stream(n, d, seed):
    return low_rank_noisy(n, d, 6, spectrum("powerlaw", 6), noise=0.05, seed=seed)


@pytest.mark.parametrize("d,ell,n,delta,seed", [(32, 4, 200, 1e-4, 2), (64, 8, 400, 1e-2, 3),
                                                (256, 80, 500, 1e-3, 4)])
def test_amplified_parity(d, ell, n, delta, seed):
    p = _gpu()
    A = _stream(n, d, seed)
    s = p.Sketch(d, ell, seed=seed, delta=delta, trace=True)
    s.update(A)
    st = s.stats()
    assert st["device_status"] == 0
    ev = s.trace()
    rep = p.binding.replay_from_trace(ev)
    o = AeroSketch(d, ell, seed=seed, delta=delta, replay=rep, tie_rel=TIE).run(A.astype(np.float64))
    assert not o.mismatches, o.mismatches[:5]
    # every doubling step the oracle amplified carries the GPU's kept SI
    amp_keys = {k for k in rep if isinstance(k, tuple)}
    assert len(amp_keys) == len(o.amp_choices) > 0
    for i, j, cs, h in o.amp_choices:
        assert rep[("amp", i, j)] == h
        assert 1 <= h <= o.amp_r
    assert st["dumps"] == len(o.S)
    assert st["shrinks"] == len(o.shrink_rows)
    AtA = A.astype(np.float64).T @ A.astype(np.float64)
    eg, eo = cov_err(A, s.query(), AtA), cov_err(A, o.query(), AtA)
    assert abs(eg - eo) <= 1e-6, (eg, eo)
    assert np.abs(s.query_gram() - o.pre_query()).max() <= 1e-5 * np.trace(AtA)
    assert eg <= 2.0 / ell


def test_r1_matches_the_plain_step_with_eps_si_02():
    """delta = 0.5: r = 1, so each amplified step is the plain step with
    eps_SI = 0.2 and the same draw; the decisions and the sketch coincide."""
    p = _gpu()
    d, ell = 48, 6
    A = _stream(300, d, 5)
    a = p.Sketch(d, ell, seed=5, delta=0.5, trace=True)
    b = p.Sketch(d, ell, seed=5, eps_si=0.2, trace=True)
    a.update(A)
    b.update(A)
    ea, eb = a.trace(), b.trace()
    assert [(e["i"], e["j_stop"], e["xi"]) for e in ea] == [(e["i"], e["j_stop"], e["xi"]) for e in eb]
    assert all(e["amp_choice"] & 15 == 1 for e in ea)
    ga, gb = a.query_gram(), b.query_gram()
    assert np.abs(ga - gb).max() <= 1e-6 * np.trace(gb)


@pytest.mark.parametrize("delta", [-0.1, 1.0, 1.5, 1e-20])
def test_delta_out_of_range(delta):
    """0 < delta < 1, and small enough counts (r <= 15, s <= 63) for the
    trace's 4-bit choices and the estimates' Philox sub-indices."""
    p = _gpu()
    with pytest.raises(p.AeroSketchError):
        p.Sketch(32, 4, delta=delta)
