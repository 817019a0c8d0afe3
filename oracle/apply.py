"""Relative Frobenius error ||A - U S V||_F / ||A||_F of a compressed matrix,
the accuracy measure of the paper's accuracy study (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np


def rel_error_dense(gen, U, s, V, row_chunk=2048, rows=None):
    """||A - U diag(s) V||_F / ||A||_F with A generated in row chunks.

    ``rows``: evaluate on these rows of A only (a sampled estimate); default
    all rows."""
    num = 0.0
    den = 0.0
    cols = np.arange(gen.n)
    allrows = np.arange(gen.m) if rows is None else np.asarray(rows)
    for r0 in range(0, allrows.size, row_chunk):
        I = allrows[r0:r0 + row_chunk]
        A = gen(I, cols)
        E = A - (U[I] * s[None, :]) @ V
        num += float(np.sum(np.abs(E) ** 2))
        den += float(np.sum(np.abs(A) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else 0.0
