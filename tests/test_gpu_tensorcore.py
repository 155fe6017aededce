"""Tensor-core (tcgen05, BF16 -> FP32 in TMEM) building block of the FD solve."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas

pytestmark = pytest.mark.gpu


def test_tcgen05_mma_selftest():
    D, timed_out = dgfas.dgfas_tc_selftest()
    assert not timed_out
    r = np.arange(128)[:, None]
    k = np.arange(16)[None, :]
    A = ((r + 2 * k) % 7 - 3).astype(np.float64)
    n = np.arange(16)[:, None]
    B = ((3 * n + k) % 5 - 2).astype(np.float64)
    np.testing.assert_array_equal(D, A @ B.T)
