"""Hierarchical-matrix use of H-BACA (argument marshalling over the C ABI).

The paper compresses one off-diagonal block of a kernel matrix whose rows and
columns have been permuted by a KD-tree partitioning (Sec. 5), and presents
H-BACA as the low-rank compression tool of hierarchical matrices (Sec. 1).
Here the KD ordering and the admissible-block partition come from the
library (hbaca_kdtree_order, hbaca_hmatrix_blocks, host C++), and all
admissible blocks of a Gaussian kernel matrix are compressed by one
hbaca_compress_batched call; the inadmissible (near-field) blocks are left
dense, as in any hierarchical matrix.
"""
import numpy as np

from . import binding as B


class HMatrix:
    """Admissible blocks of the Gaussian kernel matrix between x and y (each
    ordered by the KD tree), compressed together by one batched H-BACA call.

    Attributes: perm_x, perm_y (orderings of the input points), x, y (ordered
    points), blocks (nblocks x 5: row start, rows, column start, columns,
    admissible), adm (indices of the admissible blocks), batch (the
    binding.Batch of the admissible blocks)."""

    def __init__(self, ctx, x, y, h, leaf=256, eta=1.0, eps=1e-8, d=8, baca_leaf=512, rank_cap=256, seed=0):
        self.perm_x = B.kdtree_order(x, leaf)
        self.perm_y = B.kdtree_order(y, leaf)
        self.x = np.ascontiguousarray(np.asarray(x, np.float64)[self.perm_x])
        self.y = np.ascontiguousarray(np.asarray(y, np.float64)[self.perm_y])
        self.h = float(h)
        self.blocks = B.hmatrix_blocks(self.x, self.y, leaf, eta)
        self.adm = np.flatnonzero(self.blocks[:, 4] == 1)
        self.specs = [B.gaussian(self.x[r0:r0 + m], self.y[c0:c0 + n], self.h)
                      for (r0, m, c0, n, _) in self.blocks[self.adm]]
        self.opts = B.make_opts(eps, d, -int(baca_leaf), seed=seed, rank_cap=rank_cap, leaf_rank_cap=rank_cap)
        self.batch = B.Batch(ctx, self.specs, self.opts) if self.specs else None

    def compress(self, stream=None):
        if self.batch is not None:
            self.batch.run(stream)
        return self

    def ranks(self):
        return self.batch.ranks() if self.batch is not None else []

    def stored_entries(self):
        """Entries held: r (m + n) + r per admissible block, m n per dense one."""
        tot = 0
        ranks = dict(zip(self.adm.tolist(), self.ranks()))
        for i, (r0, m, c0, n, a) in enumerate(self.blocks):
            tot += ranks[i] * (m + n + 1) if a else m * n
        return int(tot)
