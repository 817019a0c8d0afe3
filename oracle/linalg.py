"""Dense kernels used by BACA and H-BACA, written out plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``greedy_qrcp``: column-pivoted QR read as its definition (Sec. 3.2: QRCP
  "greedily selects well-conditioned columns by examining column norms"): at
  step t every remaining candidate column is projected onto the orthogonal
  complement of the t columns already chosen (classical Gram-Schmidt applied
  twice), its residual norm is computed explicitly, and the largest one is
  chosen (lowest index on exact ties).  No norm down-dating is used.
* ``eps_rank``: r = min{k : Sigma_{k+1,k+1} < eps Sigma_{1,1}} (Sec. 2).
"""
import numpy as np


def _project_out(Q, X):
    """Residual of the columns of X after removing span(Q); two passes."""
    if Q.shape[1] == 0:
        return X.copy()
    R = X - Q @ (Q.conj().T @ X)
    R = R - Q @ (Q.conj().T @ R)
    return R


def greedy_qrcp(M, kmax, candidates=None, rank_tol=None):
    """Greedy column-pivoted QR of M (p x N).

    Parameters
    ----------
    M : (p, N) array.
    kmax : at most min(kmax, p) pivots are chosen (p bounds the rank).
    candidates : boolean mask of length N (None = all columns); only these
        columns may be chosen.
    rank_tol : if given, stop before step t when the chosen residual norm
        falls below ``rank_tol * (first residual norm)``, or when the first
        residual norm is 0 (the QR(A, eps) form of Sec. 2).

    Returns
    -------
    piv : list of chosen column indices in order.
    diag : residual norms of the chosen columns (|T_tt|).
    margins : (best - second) / best at every step (inf if a single
        candidate; 0 if best is at the rounding-noise level, below 1e-12
        times the largest initial candidate norm).
    Q : (p, len(piv)) orthonormal basis of the chosen columns (a column is
        zero when its residual norm was zero).
    """
    M = np.asarray(M)
    p, N = M.shape
    cand = np.ones(N, bool) if candidates is None else np.array(candidates, bool)
    piv, diag, margins = [], [], []
    Q = np.zeros((p, 0), dtype=np.result_type(M.dtype, np.float64))
    all_norms = np.sqrt((np.abs(M[:, cand]) ** 2).sum(axis=0))
    noise = 1e-12 * (all_norms.max() if all_norms.size else 0.0)
    for _ in range(min(kmax, p)):
        idx = np.flatnonzero(cand)
        if idx.size == 0:
            break
        R = _project_out(Q, M[:, idx])
        norms = np.sqrt((np.abs(R) ** 2).sum(axis=0))
        b = int(np.argmax(norms))
        best = norms[b]
        if rank_tol is not None:
            if len(diag) == 0 and best == 0.0:
                break
            if len(diag) > 0 and best < rank_tol * diag[0]:
                break
        if idx.size > 1:
            second = np.max(np.delete(norms, b))
            margins.append((best - second) / best if best > noise else 0.0)
        else:
            margins.append(np.inf)
        j = int(idx[b])
        piv.append(j)
        diag.append(best)
        cand[j] = False
        q = R[:, b] / best if best > 0 else np.zeros(p, dtype=Q.dtype)
        Q = np.concatenate([Q, q[:, None]], axis=1)
    return piv, diag, margins, Q


def eps_rank(s, eps):
    """eps-rank of a descending singular value list (Sec. 2)."""
    s = np.asarray(s)
    if s.size == 0 or s[0] == 0.0:
        return 0
    return int(np.count_nonzero(s >= eps * s[0]))


def truncated_svd(A, eps):
    """[U, Sigma, V, r] = SVD(A, eps) (Sec. 2): LAPACK gesdd with a gesvd
    fallback, truncated at the eps-rank.  Returns U (m x r), s (r), Vh (r x n)."""
    A = np.asarray(A)
    m, n = A.shape
    if m == 0 or n == 0:
        return (np.zeros((m, 0), A.dtype), np.zeros(0), np.zeros((0, n), A.dtype))
    try:
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
    except np.linalg.LinAlgError:
        import scipy.linalg
        U, s, Vh = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesvd")
    r = eps_rank(s, eps)
    return U[:, :r], s[:r], Vh[:r]
