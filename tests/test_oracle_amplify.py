"""Pins of the oracle's probability amplification (Algorithm 7, reading R17).

* r = 1 (delta >= 0.02): the amplified step is the plain step with
  eps_SI = 0.2 and the same random draws, so the runs coincide exactly.
* The kept simultaneous iteration is the one with the smallest estimate of
  its residual's top eigenvalue (a minimum, not a maximum or the first).
* The deterministic error bound (2/l) holds with amplification on.
"""
import numpy as np

from oracle.aerosketch import AeroSketch, default_q
from oracle.metric import cov_err
from synth import low_rank_noisy, spectrum


def _stream(n, d, seed):
    return low_rank_noisy(n, d, 6, spectrum("powerlaw", 6), noise=0.05, seed=seed).astype(np.float64)


def test_r1_is_the_plain_step_with_eps_si_02():
    d, ell = 32, 4
    A = _stream(160, d, 1)
    amp = AeroSketch(d, ell, delta=0.05).run(A)
    assert amp.amp_r == 1 and amp.amp_choices
    plain = AeroSketch(d, ell, q=default_q(d, 0.2)).run(A)
    assert len(amp.S) == len(plain.S)
    assert np.array_equal(amp.C, plain.C)
    for a, b in zip(amp.S, plain.S):
        assert a.t == b.t and np.array_equal(a.Z, b.Z)


def test_choice_minimises_the_estimates():
    d, ell = 32, 4
    A = _stream(200, d, 2)
    s = AeroSketch(d, ell, delta=1e-4).run(A)
    assert s.amp_r == 3 and s.amp_s == 19
    assert len(s.amp_choices) > 10
    for i, j, cs, h in s.amp_choices:
        assert len(cs) == 3
        assert cs[h - 1] == min(cs)
        assert all(c >= 0.0 for c in cs)


def test_amplified_error_bound():
    d, ell = 40, 5
    A = _stream(300, d, 3)
    s = AeroSketch(d, ell, delta=1e-3).run(A)
    assert cov_err(A, s.query()) <= 2.0 / ell
