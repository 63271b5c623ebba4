"""Allocation failures (AS_ENOMEM) injected through the library's test hook,
as_inject_alloc_failure: no device is driven out of memory.  Each failing call
returns AS_ENOMEM and leaves the sketch as it was; the sketch keeps working."""
import numpy as np
import pytest

from synth import low_rank_noisy, spectrum

pytestmark = pytest.mark.gpu


@pytest.fixture
def p():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    p.load_library()
    yield p
    p.lib().as_inject_alloc_failure(-1)


def _enomem(p, fn):
    with pytest.raises(p.AeroSketchError) as e:
        fn()
    assert e.value.code == p.binding.AS_ENOMEM
    p.lib().as_inject_alloc_failure(-1)


@pytest.mark.parametrize("after", [0, 3, 7])
def test_create_fails_cleanly(p, after):
    p.lib().as_inject_alloc_failure(after)
    _enomem(p, lambda: p.Sketch(64, 8))
    s = p.Sketch(64, 8)                 # the hook turned itself off
    s.update(low_rank_noisy(30, 64, 4, spectrum("geometric", 4), seed=1))
    assert s.stats()["device_status"] == 0


@pytest.mark.parametrize("dense", [False, True])
def test_query_failure_leaves_the_sketch(p, dense):
    d, ell = 256, 16
    A = low_rank_noisy(120, d, 8, spectrum("geometric", 8), seed=2)
    s = p.Sketch(d, ell, dense_query=dense)
    s.update(A)
    B0, Bh0 = s.query_gram(), s.query()
    for after in (0, 2, 4):     # every route makes at least five allocations
        p.lib().as_inject_alloc_failure(after)
        _enomem(p, lambda: s.query())
        assert np.array_equal(s.query_gram(), B0)
        assert np.array_equal(s.query(), Bh0)
    s.update(A[:10])
    assert s.stats()["rows"] == 130


def test_reserve_and_merge_failures(p):
    d, ell = 128, 8
    A = low_rank_noisy(200, d, 6, spectrum("geometric", 6), seed=3)
    s1, s2 = p.Sketch(d, ell, seed=1), p.Sketch(d, ell, seed=2)
    s1.update(A[:100])
    s2.update(A[100:])
    g1 = s1.query_gram()
    p.lib().as_inject_alloc_failure(0)
    _enomem(p, lambda: s1.reserve(1000))
    p.lib().as_inject_alloc_failure(0)
    _enomem(p, lambda: s1.merge(s2))
    assert np.array_equal(s1.query_gram(), g1)
    s1.merge(s2)
    assert np.abs(s1.query_gram() - (g1 + s2.query_gram())).max() <= 1e-12 * np.trace(g1)


def test_hook_rejects_bad_argument(p):
    assert p.lib().as_inject_alloc_failure(-2) == p.binding.AS_EINVAL
