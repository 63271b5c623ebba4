"""The tcgen05 GEMM (through the C ABI) against an FP64 product of the same operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_02019_gb300 as p
    return p


def _bf16(x):
    """Round FP32 to BF16 (nearest even) and back, in numpy."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("M,N,K,splits", [(128, 32, 64, 1), (300, 70, 200, 1), (1000, 192, 2048, 4),
                                          (2048, 64, 4096, 8), (64, 256, 128, 1), (129, 17, 520, 3)])
def test_bf16_single_pass_exact_products(M, N, K, splits):
    """npass = 1: the result equals the FP64 product of the BF16-rounded operands
    up to FP32 accumulation error."""
    p = _p()
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    got = p.binding.tc_gemm(A, B, npass=1, splits=splits)
    ref = _bf16(A).astype(np.float64) @ _bf16(B).astype(np.float64).T
    tol = 1e-5 * np.sqrt(K) * np.abs(ref).max() / np.sqrt(K) + 1e-6 * np.sqrt(K)
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("M,N,K,splits", [(256, 128, 1024, 2), (2048, 192, 2048, 10)])
def test_split_bf16_is_near_fp32(M, N, K, splits):
    """npass = 3: hi*hi + hi*lo + lo*hi reaches ~2^-16 relative per product."""
    p = _p()
    rng = np.random.default_rng(7)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    got = p.binding.tc_gemm(A, B, npass=3, splits=splits)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    err1 = np.abs(p.binding.tc_gemm(A, B, npass=1, splits=splits) - ref).max()
    err3 = np.abs(got - ref).max()
    assert err3 <= 1e-4 * np.sqrt(K)
    assert err3 < err1 / 50


def test_three_level_split_is_fp32_accurate():
    """npass = 6: the three-level split reaches FP32-product accuracy."""
    p = _p()
    rng = np.random.default_rng(11)
    A = rng.standard_normal((512, 1024)).astype(np.float32)
    B = rng.standard_normal((96, 1024)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    err6 = np.abs(p.binding.tc_gemm(A, B, npass=6, splits=4) - ref).max()
    err3 = np.abs(p.binding.tc_gemm(A, B, npass=3, splits=4) - ref).max()
    assert err6 <= 1e-4 * np.sqrt(1024)
    assert err6 < err3
