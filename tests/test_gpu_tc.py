"""Tensor-core self-test: the operand layout and the exact integer
accumulation that the tensor-core split-precision half-step relies on."""
import numpy as np
import pytest

from tests.gpu_util import lib_built, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


@pytest.mark.parametrize("K,N", [(16, 32), (64, 48), (128, 96), (112, 80)])
def test_tc_selftest_exact_integer_products(hb, K, N):
    A = np.zeros((128, K), np.float32)
    B = np.zeros((N, K), np.float32)
    D0 = np.zeros((128, N), np.float32)
    D1 = np.zeros((128, N - 16), np.float32)
    rc = hb.lib().hermite_tc_selftest(K, N, A.ctypes.data, B.ctypes.data, D0.ctypes.data, D1.ctypes.data)
    assert rc == 0
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.abs(ref).max() < 2**24 and np.abs(ref).max() > 0.3 * K * 2**16  # large sums are exercised
    np.testing.assert_array_equal(D0.astype(np.int64), ref)
    np.testing.assert_array_equal(D1.astype(np.int64), ref[:, : N - 16])
