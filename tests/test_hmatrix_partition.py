"""KD ordering and admissible-block partition (host C++ through the C ABI; no
GPU): a permutation whose index-tree nodes are spatial cells, blocks that tile
the matrix, and the admissibility condition min(diam) <= eta dist."""
import numpy as np
import pytest

from paper_1901_06101_gb300 import binding as B


@pytest.fixture(scope="module")
def lib():
    try:
        return B.lib()
    except RuntimeError:
        pytest.skip("libhbaca.so not built")


def _box(P):
    return P.min(axis=0), P.max(axis=0)


def test_kdtree_order_cells_are_split_along_the_widest_side(lib):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3000, 3)) * np.array([4.0, 1.0, 0.5])
    p = B.kdtree_order(x, 100)
    assert np.array_equal(np.sort(p), np.arange(3000))
    xo = x[p]

    def check(s0, s):
        if s <= 100:
            return
        lo, hi = _box(xo[s0:s0 + s])
        k = int(np.argmax(hi - lo))
        a = (s + 1) // 2
        assert xo[s0:s0 + a, k].max() <= xo[s0 + a:s0 + s, k].min()
        check(s0, a)
        check(s0 + a, s - a)
    check(0, 3000)


@pytest.mark.parametrize("eta", [0.5, 1.0, 2.0])
def test_hmatrix_blocks_tile_and_are_admissible(lib, eta):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (2000, 3))
    y = rng.uniform(0, 1, (1500, 3)) + np.array([0.5, 0.0, 0.0])
    xo, yo = x[B.kdtree_order(x, 64)], y[B.kdtree_order(y, 64)]
    bl = B.hmatrix_blocks(xo, yo, 64, eta)
    cover = np.zeros((2000, 1500), np.int32)
    for r0, m, c0, n, adm in bl:
        cover[r0:r0 + m, c0:c0 + n] += 1
        (lx, hx), (ly, hy) = _box(xo[r0:r0 + m]), _box(yo[c0:c0 + n])
        diam = min(np.linalg.norm(hx - lx), np.linalg.norm(hy - ly))
        dist = np.linalg.norm(np.maximum(0.0, np.maximum(ly - hx, lx - hy)))
        if adm:
            assert diam <= eta * dist * (1 + 1e-12)
        else:
            assert m <= 64 and n <= 64
    assert np.all(cover == 1)
    assert bl[:, 4].sum() > 0
