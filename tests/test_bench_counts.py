"""Work counts the benchmark divides by the QR and Q-application times: the
closed forms against the flops of the Householder loops counted entry by
entry (CPU only)."""
import numpy as np
import pytest

import bench


def _qr_loop(m, k):
    # reflector j (m - j rows) applied to the k - j - 1 trailing columns:
    # inner product and update, two flops per entry each
    return sum(4 * (m - j) * (k - j - 1) for j in range(min(k, m)))


def _qapply_loop(m, k, s):
    # reflector j touches rows j .. m-1 of each of the s columns: inner
    # product and update, two flops per entry each
    return sum(4 * (m - j) * s for j in range(k))


@pytest.mark.parametrize("m,k", [(1250, 113), (4000, 400), (20000, 132), (300, 300)])
def test_qr_count_leading_order(m, k):
    brute = _qr_loop(m, k)
    assert abs(bench.qr_flops(m, k) / brute - 1.0) < 3.0 / min(k, m)


@pytest.mark.parametrize("m,k,s", [(1250, 113, 66), (20000, 132, 66), (64, 64, 1)])
def test_qapply_count_leading_order(m, k, s):
    brute = _qapply_loop(m, k, s)
    assert abs(bench.qapply_flops(m, k, s) / brute - 1.0) < 1.0 / m


def test_dense_flops_sides():
    # one leaf task (both factors, both applications) and one merge task
    # (stacked side only); complex doubles the count twice
    leaf = np.array([[113, 113, 113, 66, 7, 66, 0, 0]], np.int32)
    merge = np.array([[132, 132, 0, 66, 7, 66, 0, 0]], np.int32)
    dims = [(0, leaf, np.array([1250]), np.array([1000])), (1, merge, np.array([2500]), np.array([0]))]
    qr, qa = bench.dense_flops(dims, False)
    assert qr == pytest.approx(bench.qr_flops(1250, 113) + bench.qr_flops(1000, 113) + bench.qr_flops(2500, 132))
    assert qa == pytest.approx(bench.qapply_flops(1250, 113, 66) + bench.qapply_flops(1000, 113, 66)
                               + bench.qapply_flops(2500, 132, 66))
    qr4, qa4 = bench.dense_flops(dims, True)
    assert (qr4, qa4) == pytest.approx((4 * qr, 4 * qa))
