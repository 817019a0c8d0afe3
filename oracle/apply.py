"""Application of the compressed operator, y = U (S (V X)), and the dense
relative Frobenius error ||A - U S V||_F / ||A||_F used by the accuracy
study (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np


def apply(U, s, V, X):
    """y = U diag(s) V X."""
    return U @ (s[:, None] * (V @ X))


def rel_error_dense(gen, U, s, V, row_chunk=2048):
    """||A - U S V||_F / ||A||_F with A generated in row chunks."""
    num = 0.0
    den = 0.0
    cols = np.arange(gen.n)
    for r0 in range(0, gen.m, row_chunk):
        I = np.arange(r0, min(gen.m, r0 + row_chunk))
        A = gen(I, cols)
        E = A - (U[I] * s[None, :]) @ V
        num += float(np.sum(np.abs(E) ** 2))
        den += float(np.sum(np.abs(A) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else 0.0
