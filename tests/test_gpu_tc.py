"""Tensor-core probe (tcgen05.mma kind::f16, accumulator in tensor memory):
products of 8-bit integers held in f16 and their f32 sums must be exact, for
the operand layout the base-conversion kernels use.  Compared with an int64
matrix product computed here."""
import numpy as np
import pytest

from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return hp.load()


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("n", [256, 208, 112, 16])
def test_tc_gemm_exact_random_limbs(n, bf16):
    rng = np.random.default_rng(n)
    A = rng.integers(0, 256, (128, 112))
    B = rng.integers(0, 256, (n, 112))
    D = hp.probe_tc_gemm(A, B, bf16=bf16)
    assert np.array_equal(D.astype(np.int64), A @ B.T)


@pytest.mark.parametrize("bf16", [False, True])
def test_tc_gemm_exact_at_the_largest_sums(bf16):
    """112 products of 255 x 255: 7,282,800 < 2^23, still exact in f32."""
    A = np.full((128, 112), 255)
    B = np.full((208, 112), 255)
    B[5, :] = np.arange(112) % 256
    D = hp.probe_tc_gemm(A, B, bf16=bf16)
    assert np.array_equal(D.astype(np.int64), A @ B.T)


def test_tc_gemm_structured_positions():
    """Distinct values per (row, k) expose any mix-up of the operand layout."""
    A = (np.arange(128)[:, None] * 3 + np.arange(112)[None, :] * 5) % 251
    B = (np.arange(256)[:, None] * 7 + np.arange(112)[None, :] * 11) % 241
    for bf16 in (False, True):
        D = hp.probe_tc_gemm(A, B, bf16=bf16)
        assert np.array_equal(D.astype(np.int64), A @ B.T)


def test_bounded_wait_expires_without_fault():
    """No MMA is issued, so the mbarrier never completes: the kernel's bounded
    wait expires, it reports HP_ERR_TIMEOUT through its status word, frees its
    tensor memory, and the device keeps working (a product right after is exact)."""
    lib = hp.load()
    assert lib.hp_probe_tc_timeout(1024) == hp.HP_ERR_TIMEOUT
    assert lib.hp_probe_tc_timeout(0) == hp.HP_ERR_ARG
    A = np.full((128, 112), 3)
    B = np.full((16, 112), 5)
    assert np.array_equal(hp.probe_tc_gemm(A, B).astype(np.int64), A @ B.T)
