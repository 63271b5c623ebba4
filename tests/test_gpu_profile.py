"""The kernel-class profiler (AS_PROFILE) and its class selection.

A library service with no counterpart in the paper: timing a subset of the
classes keeps the other classes' event records off the update path.  Timing
must not change what the sketch computes.
"""
import numpy as np
import pytest

import paper_2601_02019_gb300 as p
from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu


def _rows(n=600, d=256):
    return low_rank_noisy(n, d, 12, spectrum("powerlaw", 12), stream=3)


@pytest.mark.parametrize("prec", [0, 3])
def test_profile_select_times_only_the_chosen_classes(prec):
    A = _rows()
    plain = p.Sketch(256, 64, prec=prec)   # fed in the same two calls
    plain.update(A[:300])
    plain.update(A[300:])
    prof = p.Sketch(256, 64, prec=prec, profile=True)
    prof.update(A[:300])
    full = {k["name"]: k["launches"] for k in prof.profile()}
    assert full["ingest"] > 0 and full["gram_rows_gemm"] > 0
    chosen = ["ingest", "eig_tridiag"]
    prof.profile_select(chosen)
    prof.profile_reset()
    prof.update(A[300:])
    after = {k["name"]: k["launches"] for k in prof.profile()}
    assert after["ingest"] > 0
    assert all(v == 0 for name, v in after.items() if name not in chosen), after
    # the timing does not change the sketch
    C0, r0 = plain.buffer()
    C1, r1 = prof.buffer()
    assert r0 == r1
    assert np.array_equal(C0, C1)
    with pytest.raises(ValueError):
        prof.profile_select(["no_such_class"])
    prof.profile_select(None)
