"""as_symeig_noalloc: the eigensolver entry point that allocates nothing.

It serves callers that cannot allocate device memory (allocator callbacks,
real-time serving loops that forbid allocation after start-up).  Its output must equal that of as_symeig, which
allocates its own buffers, on consecutive calls that share the library's
fixed scratch array.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    return p, torch


def _noalloc(p, torch, A, nev):
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dl = torch.zeros(nev, dtype=torch.float64, device="cuda")
    dV = torch.zeros((n, nev), dtype=torch.float64, device="cuda")
    code = p.lib().as_symeig_noalloc(n, ct.c_void_p(dA.data_ptr()), nev, ct.c_void_p(dl.data_ptr()),
                                     ct.c_void_p(dV.data_ptr()), None)
    assert code == 0, p.lib().as_status_str(code)
    torch.cuda.synchronize()
    return dl.cpu().numpy(), dV.cpu().numpy()


def test_matches_allocating_entry_point_on_consecutive_calls():
    p, torch = _setup()
    rng = np.random.default_rng(3)
    # calls in a row share the scratch array; (128, 128) is the largest order,
    # where the copy of A and the solver's work fill the array exactly
    for n, nev in [(100, 40), (64, 64), (128, 128)]:
        B = rng.standard_normal((n, n + 5))
        A = B @ B.T
        lam0, V0 = p.binding.symeig(A, nev)
        lam1, V1 = _noalloc(p, torch, A, nev)
        scale = np.abs(lam0).max()
        assert np.abs(lam1 - lam0).max() <= 1e-11 * scale
        # eigenvectors agree up to sign (the spectrum here is simple)
        dots = np.abs(np.sum(V0 * V1, axis=0))
        assert np.abs(dots - 1.0).max() <= 1e-8


def test_rejects_orders_beyond_the_scratch_size():
    p, torch = _setup()
    dA = torch.zeros((129, 129), dtype=torch.float64, device="cuda")
    dl = torch.zeros(1, dtype=torch.float64, device="cuda")
    dV = torch.zeros((129, 1), dtype=torch.float64, device="cuda")
    code = p.lib().as_symeig_noalloc(129, ct.c_void_p(dA.data_ptr()), 1, ct.c_void_p(dl.data_ptr()),
                                     ct.c_void_p(dV.data_ptr()), None)
    assert code == p.binding.AS_EINVAL
