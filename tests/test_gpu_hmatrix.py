"""Hierarchical-matrix use of the batched H-BACA path (Sec. 1: H-BACA as the
compression tool of hierarchical matrices; Sec. 5: rows and columns permuted
by a KD tree).  Needs a GB300."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import generators as og
from oracle import hbaca as oh
from paper_1901_06101_gb300 import binding as B
from paper_1901_06101_gb300 import hmatrix
from paper_1901_06101_gb300 import inputs
from tests.test_gpu_batched import levels_for
from tests.test_gpu_parity import check_result, compare_with_frozen_oracle, run_and_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return B.Context()


def test_admissible_blocks_of_a_gaussian_hmatrix(ctx):
    """All admissible blocks of the Gaussian kernel matrix of 12000 points in
    the unit cube (KD leaves of 200 points, eta = 1) compressed by one batched
    call: eight blocks against the frozen-pivot oracle H-BACA (batch index =
    block number), and the whole hierarchical matrix (low-rank blocks plus
    dense near field) against the dense matrix on 300 sampled rows."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0.0, 1.0, (12000, 3))
    h, eps, d, target = 0.25, 1e-8, 8, 256
    H = hmatrix.HMatrix(ctx, x, x, h, leaf=200, eta=1.0, eps=eps, d=d, baca_leaf=target, rank_cap=256)
    H.compress()
    torch.cuda.synchronize()
    assert len(H.adm) >= 50
    res = H.batch.results()
    sizes = H.blocks[H.adm][:, [1, 3]]
    pick = sorted(set(np.linspace(0, len(H.adm) - 1, 8).astype(int).tolist()))
    for b in pick:
        r0, m, c0, n, _ = H.blocks[H.adm[b]]
        ogen = og.Gaussian(H.x[r0:r0 + m], H.y[c0:c0 + n], h)
        L = levels_for(m, n, target)
        traces = {leaf: B.read_leaf_trace_batched(H.specs, H.opts, H.batch.ws, b, leaf) for leaf in range(4 ** L)}
        full = oh.hbaca(ogen, L, d, eps, seed=0, batch_index=b, forced=traces)
        check_result(ogen, res[b], eps, full)
    # the assembled hierarchical matrix on sampled rows
    gen = og.Gaussian(H.x, H.y, h)
    rows = np.sort(rng.choice(12000, 300, replace=False))
    approx = np.zeros((rows.size, 12000))
    adm_of = {int(i): k for k, i in enumerate(H.adm)}
    for i, (r0, m, c0, n, a) in enumerate(H.blocks):
        sel = np.flatnonzero((rows >= r0) & (rows < r0 + m))
        if sel.size == 0:
            continue
        if a:
            c = res[adm_of[i]]
            U, S, V = c.U.cpu().numpy(), c.S.cpu().numpy(), c.V.cpu().numpy()
            approx[sel, c0:c0 + n] = (U[rows[sel] - r0] * S) @ V
        else:
            approx[sel, c0:c0 + n] = gen(rows[sel], np.arange(c0, c0 + n))
    A = gen(rows, np.arange(12000))
    err = np.linalg.norm(A - approx) / np.linalg.norm(A)
    assert err <= 2 * eps, err
    ranks = H.ranks()
    print("H-matrix 12000: %d blocks, %d admissible (sizes %d-%d), ranks %d-%d, stored %.1f%% of dense, "
          "sampled-row error %.2e" % (len(H.blocks), len(H.adm), sizes.min(), sizes.max(), min(ranks), max(ranks),
                                      100.0 * H.stored_entries() / 12000 ** 2, err))


def test_kdtree_ordering_lowers_leaf_ranks(ctx):
    """The benchmark's Helmholtz geometry at 8000^2 (8 x 8 leaves): with both
    point sets in KD order every leaf is a pair of spatial cells and its BACA
    rank falls well below that of the drawn order, while the compressed matrix
    (the same matrix, permuted) keeps its rank and error; the ordered run
    matches the frozen-pivot oracle."""
    x, y = inputs.sphere_pair(seed=1, m=8000, n=8000)
    k, eps, d, L = 4 * np.pi, 1e-4, 16, 3
    px, py = B.kdtree_order(x, 1000), B.kdtree_order(y, 1000)
    xo, yo = x[px], y[py]
    plain = B.compress(ctx, B.helmholtz(x, y, k), B.make_opts(eps, d, L, seed=1, rank_cap=256, leaf_rank_cap=256))
    spec = B.helmholtz(xo, yo, k)
    ogen = og.Helmholtz(xo, yo, k)
    res, compared, div, tr = run_and_compare(ctx, spec, ogen, L, d, eps, seed=1, rank_cap=256, leaf_cap=256,
                                             check_all_leaves=False)
    opts = B.make_opts(eps, d, L, seed=1, rank_cap=256, leaf_rank_cap=256)
    tr = {leaf: B.read_leaf_trace(spec, opts, res.ws, leaf) for leaf in range(64)}
    full = oh.hbaca(ogen, L, d, eps, seed=1, forced=tr)
    compare_with_frozen_oracle(res, full, ogen, tr)
    assert abs(res.rank - plain.rank) <= 2
    assert res.res.leaf_rank_max < 0.8 * plain.res.leaf_rank_max, (res.res.leaf_rank_max, plain.res.leaf_rank_max)
    print("KD order: leaf BACA rank max %d (drawn order %d); final rank %d (%d)"
          % (res.res.leaf_rank_max, plain.res.leaf_rank_max, res.rank, plain.rank))
