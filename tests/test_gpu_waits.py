"""The library's bounded device waits (release flags, grid barriers, mbarrier
phases) give up as designed.

Each self-test kernel waits on something that nothing completes, with a
100 ms limit in place of the production 2 s.  The wait must end, the call must
report AS_ETIMEOUT, and the context must still run a sketch afterwards.  No
GPU fault is involved: the waits return on their own.
"""
import time

import numpy as np
import pytest

from synth import low_rank_noisy, spectrum


def _lib():
    import paper_2601_02019_gb300 as p
    try:
        p.load_library()
    except Exception as e:   # pragma: no cover - library not built
        pytest.skip(str(e))
    return p


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_bounded_wait_gives_up_and_the_context_survives(kind):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = _lib()
    t0 = time.perf_counter()
    code = p.lib().as_wait_selftest(kind, 100, None)
    dt = time.perf_counter() - t0
    assert code == p.binding.AS_ETIMEOUT
    assert 0.1 <= dt < 5.0, dt
    s = p.Sketch(32, 4)
    s.update(low_rank_noisy(60, 32, 4, spectrum("geometric", 4), seed=1))
    assert s.stats()["device_status"] == 0


def test_selftest_rejects_bad_arguments():
    """Argument checks happen on the host, before any device call."""
    p = _lib()
    for kind, ms in [(-1, 100), (3, 100), (0, 0), (0, 2001)]:
        assert p.lib().as_wait_selftest(kind, ms, None) == p.binding.AS_EINVAL
