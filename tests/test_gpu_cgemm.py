"""The tensor-core complex GEMM (tcgen05, 3xTF32) against a complex128 product."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


@pytest.mark.parametrize("shape", [(1, 128, 128, 32), (3, 200, 77, 45), (2, 64, 300, 96), (1, 512, 558, 512),
                                   (2, 5, 3, 1)])
def test_cgemm_matches_fp64_product(pw, shape):
    b, M, N, K = shape
    rng = np.random.default_rng(sum(shape))
    A = (rng.standard_normal((b, M, K)) + 1j * rng.standard_normal((b, M, K))).astype(np.complex64)
    B = (rng.standard_normal((b, K, N)) + 1j * rng.standard_normal((b, K, N))).astype(np.complex64)
    C = (rng.standard_normal((b, M, N)) + 1j * rng.standard_normal((b, M, N))).astype(np.complex64)
    got = pw.cgemm_c64(A, B, C)
    ref = C.astype(np.complex128) - A.astype(np.complex128) @ B.astype(np.complex128)
    # 3xTF32 products; the tensor cores' FP32 accumulation truncates, so the kernel
    # restarts it every 32-complex K stage and sums the stages in FP32 registers:
    # truncation accrues over at most 24 MMAs (3 x 8 per stage), ~24 * 2^-24.
    scale = np.sqrt(K) * 2.0
    err = np.max(np.abs(got - ref)) / scale
    print(f"cgemm {shape}: max error / (2 sqrt K) = {err:.2e}")
    assert err < 4.0 * 24 * 2.0 ** -24 * max(1.0, np.sqrt(K / 32.0)), err
