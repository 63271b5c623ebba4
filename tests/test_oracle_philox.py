"""Pins of the oracle's Philox4x64-10 and Box-Muller against independent sources."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox


@pytest.mark.parametrize("key", [(0, 0), (12345, 678), (2**64 - 1, 2**63 + 5)])
@pytest.mark.parametrize("ctr0", [0, 5, 2**40 + 3])
def test_matches_numpy_philox(key, ctr0):
    # numpy's Philox bit generator (an independent implementation of the same
    # published generator) bumps the counter before producing each 4-word block.
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64))
    st = bg.state
    st["state"]["counter"] = np.array([ctr0, 7, 9, 11], dtype=np.uint64)
    st["buffer_pos"] = 4
    bg.state = st
    raw = bg.random_raw(12).reshape(3, 4)
    ctr = np.array([[ctr0 + 1 + b, 7, 9, 11] for b in range(3)], dtype=np.uint64)
    mine = philox.philox4x64_10(ctr, key)
    assert np.array_equal(raw, mine)


def test_uniform_open_interval():
    w = np.array([0, 2**64 - 1, 2**12 - 1, 2**12], dtype=np.uint64)
    u = philox.uniform53(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[1] == 1.0 - 2.0**-53
    assert u[0] == 0.5 * 2.0**-52 and u[2] == u[0] and u[3] == 1.5 * 2.0**-52


def test_gaussians_are_standard_normal():
    z = philox.gaussians(3, 1, philox.PURPOSE_PI_START, 17, 0, 200_000)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.02
    # lanes are independent: lag-1 correlation ~ 0
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 0.01


def test_gaussians_counter_layout():
    # element e comes from counter block e >> 2, so a prefix is stable and
    # different (purpose, i, j) give different streams
    a = philox.gaussians(0, 0, 4, 10, 2, 64)
    b = philox.gaussians(0, 0, 4, 10, 2, 7)
    assert np.array_equal(a[:7], b)
    c = philox.gaussians(0, 0, 4, 10, 3, 64)
    assert not np.allclose(a, c)
