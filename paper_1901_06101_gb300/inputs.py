"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module draws points, sparse factors and right-hand sides only.  It holds
none of the compression method's arithmetic, so both the CUDA path and the
CPU checker can be fed from it.  The paper's data sets (UCI SUSY / MNIST
features, EFIE meshes, multifrontal fronts) are not available; these draws
stand in for them.

Workloads (sizes and distributions as the benchmark configurations state):
  gaussian_pair      x ~ U[0,1]^3, y ~ U[2,3] x U[0,1]^2           (Gaussian kernel)
  sphere_pair        x uniform on the unit sphere at 0, y on the unit sphere
                     at (3, 0, 0) (normalised Gaussian draws)       (Helmholtz kernel)
  sparse_product     P (m x K) with exactly `nnz` nonzeros per column, Q (K x n)
                     with exactly `nnz` nonzeros per row, N(0,1) values; dense
                     P2 (m x 5), Q2 (5 x n) with N(0, std2^2) entries
  batched_blocks     per block: m, n log-uniform in [64, 2048]; x ~ U[0,1]^3;
                     y = U[0,1]^3 cube shifted by a distance U[2,4] along a
                     random unit direction; h log-uniform in [0.1, 10]
  lowrank            U (m x r), V (r x n) with i.i.d. N(0,1) entries
  polynomial_pair    x_i, y_j i.i.d. N(0, 1/dim) in R^dim            (polynomial kernel)
  strips_pair        n points on each of two parallel 2-D strips of length 1,
                     1 apart (segment midpoints), k = 2 pi n / 15 (15 points
                     per wavelength)                                 (EFIE2D kernel)
Points are returned in the order drawn (no spatial permutation).
"""
import numpy as np


def gaussian_pair(seed=0, m=2000, n=2000):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (m, 3))
    y = rng.uniform(0.0, 1.0, (n, 3))
    y[:, 0] += 2.0
    return x, y


def _sphere(rng, n, centre):
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g + np.asarray(centre, np.float64)[None, :]


def sphere_pair(seed=1, m=20000, n=20000):
    rng = np.random.default_rng(seed)
    x = _sphere(rng, m, (0.0, 0.0, 0.0))
    y = _sphere(rng, n, (3.0, 0.0, 0.0))
    return x, y


class SparseProductInputs:
    """CSR P, CSC Q (int32 indices, sorted within a row / column) and dense P2, Q2."""

    def __init__(self, m, n, K, p_rowptr, p_colidx, p_val, q_colptr, q_rowidx, q_val, P2, Q2):
        self.m, self.n, self.K = m, n, K
        self.p_rowptr, self.p_colidx, self.p_val = p_rowptr, p_colidx, p_val
        self.q_colptr, self.q_rowidx, self.q_val = q_colptr, q_rowidx, q_val
        self.P2, self.Q2 = P2, Q2

    def dense_P(self):
        P = np.zeros((self.m, self.K))
        for i in range(self.m):
            s, e = self.p_rowptr[i], self.p_rowptr[i + 1]
            P[i, self.p_colidx[s:e]] = self.p_val[s:e]
        return P

    def dense_Q(self):
        Q = np.zeros((self.K, self.n))
        for j in range(self.n):
            s, e = self.q_colptr[j], self.q_colptr[j + 1]
            Q[self.q_rowidx[s:e], j] = self.q_val[s:e]
        return Q


def _to_compressed(major_len, minor_idx_per_minor, vals_per_minor, n_minor):
    """Build a compressed (CSR-like) structure indexed by the major dimension
    from per-minor lists of major indices."""
    counts = np.zeros(major_len + 1, np.int64)
    for k in range(n_minor):
        np.add.at(counts, minor_idx_per_minor[k] + 1, 1)
    ptr = np.cumsum(counts)
    idx = np.empty(ptr[-1], np.int32)
    val = np.empty(ptr[-1], np.float64)
    fill = ptr[:-1].copy()
    for k in range(n_minor):  # k ascending, so indices within a major row are sorted
        rows = minor_idx_per_minor[k]
        pos = fill[rows]
        idx[pos] = k
        val[pos] = vals_per_minor[k]
        fill[rows] += 1
    return ptr.astype(np.int32), idx, val


def sparse_product(seed=2, m=50000, n=50000, K=50, density=0.01, r2=5, std2=1e-3):
    rng = np.random.default_rng(seed)
    nnz_p = int(round(density * m))
    nnz_q = int(round(density * n))
    p_rows = [np.sort(rng.choice(m, nnz_p, replace=False)) for _ in range(K)]
    p_vals = [rng.standard_normal(nnz_p) for _ in range(K)]
    q_cols = [np.sort(rng.choice(n, nnz_q, replace=False)) for _ in range(K)]
    q_vals = [rng.standard_normal(nnz_q) for _ in range(K)]
    p_rowptr, p_colidx, p_val = _to_compressed(m, p_rows, p_vals, K)
    q_colptr, q_rowidx, q_val = _to_compressed(n, q_cols, q_vals, K)
    P2 = rng.standard_normal((m, r2)) * std2
    Q2 = rng.standard_normal((r2, n)) * std2
    return SparseProductInputs(m, n, K, p_rowptr, p_colidx, p_val,
                               q_colptr, q_rowidx, q_val, P2, Q2)


def batched_blocks(seed=3, nblocks=4096, lo=64, hi=2048):
    """List of (x, y, h) Gaussian-kernel blocks."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nblocks):
        m = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        x = rng.uniform(0.0, 1.0, (m, 3))
        direction = rng.standard_normal(3)
        direction /= np.linalg.norm(direction)
        dist = rng.uniform(2.0, 4.0)
        y = rng.uniform(0.0, 1.0, (n, 3)) + dist * direction[None, :]
        h = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        out.append((x, y, h))
    return out


def grad_blocks(seed=5, nblocks=256, lo=256, hi=2048, h=0.7):
    """List of (x, y, h) Gaussian-kernel blocks shaped like the differentiated
    workload: x uniform in [0,1]^3, y uniform in [2,3]x[0,1]^2, sizes
    log-uniform in [lo, hi], one width h."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nblocks):
        m = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        x = rng.uniform(0.0, 1.0, (m, 3))
        y = rng.uniform(0.0, 1.0, (n, 3))
        y[:, 0] += 2.0
        out.append((x, y, float(h)))
    return out


def lowrank(seed, m, n, r, complex_=False):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if complex_:
        U = U + 1j * rng.standard_normal((m, r))
        V = V + 1j * rng.standard_normal((r, n))
    return U, V


def rhs(seed, n, nrhs):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, nrhs))


def polynomial_pair(seed=4, m=2000, n=2000, dim=50):
    """Random data points for the polynomial kernel: entries N(0, 1/dim), so
    that x_i^t y_j is O(1)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((m, dim)) / np.sqrt(dim)
    y = rng.standard_normal((n, dim)) / np.sqrt(dim)
    return x, y


def strips_pair(n=2000):
    """Discretisation points of two parallel strips of length 1 at distance
    1 (the EFIE2D geometry): midpoints of n equal segments of [0,1] x {0}
    and of [0,1] x {1}, and the wavenumber giving 15 points per wavelength,
    k = 2 pi n / 15."""
    t = (np.arange(n) + 0.5) / n
    x = np.stack([t, np.zeros(n)], axis=1)
    y = np.stack([t, np.ones(n)], axis=1)
    return x, y, 2.0 * np.pi * n / 15.0
