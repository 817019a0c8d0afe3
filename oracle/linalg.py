"""Dense kernels used by BACA and H-BACA, written out plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``greedy_qrcp``: column-pivoted QR read as its definition (Sec. 3.2: QRCP
  "greedily selects well-conditioned columns by examining column norms"): at
  step t every remaining candidate column is projected onto the orthogonal
  complement of the t columns already chosen (classical Gram-Schmidt applied
  twice), its residual norm is computed explicitly, and the largest one is
  chosen (lowest index on exact ties).  No norm down-dating is used.
* ``strong_rrqr``: Gu and Eisenstat's swap refinement of a chosen set, one of
  the subset-selection alternatives to QRCP that Sec. 3.2 names.
* ``eps_rank``: r = min{k : Sigma_{k+1,k+1} < eps Sigma_{1,1}} (Sec. 2).
* ``frob_rank``: the Frobenius reading of a truncation, the smallest t whose
  discarded tail sqrt(sum_{j>t} Sigma_jj^2) is at most eps_loc ||A||_F (the
  paper measures accuracy as the relative Frobenius error, Sec. 5.2).
"""
import numpy as np
import scipy.linalg


def _project_out(Q, X):
    """Residual of the columns of X after removing span(Q); two passes."""
    if Q.shape[1] == 0:
        return X.copy()
    R = X - Q @ (Q.conj().T @ X)
    R = R - Q @ (Q.conj().T @ R)
    return R


def greedy_qrcp(M, kmax, candidates=None, rank_tol=None, abs_noise=0.0, forced=None):
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
    abs_noise : absolute rounding-noise level of the residual norms; a step
        whose best-minus-second gap is below it gets margin 0.
    forced : replay mode.  The pivots are taken from this list (its length is
        the pivot count, rank_tol is not applied) and every step records
        whether the forced column is a valid greedy choice, i.e. its
        residual norm is within 1e-9 * best + abs_noise of the largest one.

    Returns
    -------
    piv : list of chosen column indices in order.
    diag : residual norms of the chosen columns (|T_tt|).
    margins : (best - second) / best at every step (inf if a single
        candidate; 0 if best is at the rounding-noise level, below 1e-12
        times the largest initial candidate norm).
    Q : (p, len(piv)) orthonormal basis of the chosen columns (a column is
        zero when its residual norm was zero).
    In replay mode a fifth element lists the validity of every forced step.
    """
    M = np.asarray(M)
    p, N = M.shape
    cand = np.ones(N, bool) if candidates is None else np.array(candidates, bool)
    piv, diag, margins = [], [], []
    Q = np.zeros((p, 0), dtype=np.result_type(M.dtype, np.float64))
    all_norms = np.sqrt((np.abs(M[:, cand]) ** 2).sum(axis=0))
    noise = max(1e-12 * (all_norms.max() if all_norms.size else 0.0), abs_noise)
    valid = []
    steps = min(kmax, p) if forced is None else len(forced)
    for step in range(steps):
        idx = np.flatnonzero(cand)
        if idx.size == 0:
            break
        R = _project_out(Q, M[:, idx])
        norms = np.sqrt((np.abs(R) ** 2).sum(axis=0))
        b = int(np.argmax(norms))
        if forced is not None:
            top = norms[b]
            hit = np.flatnonzero(idx == forced[step])
            if hit.size == 0:
                valid.append(False)
                break
            b = int(hit[0])
            ok = bool(norms[b] >= top - 1e-9 * top - noise)
            valid.append(ok if ok else (step, float(top), float(norms[b]), float(noise)))
        best = norms[b]
        if rank_tol is not None and forced is None:
            if len(diag) == 0 and best == 0.0:
                break
            if len(diag) > 0 and best < rank_tol * diag[0]:
                break
        if idx.size > 1:
            second = np.max(np.delete(norms, b))
            gap = best - second
            margins.append(gap / best if (best > noise and gap > noise) else 0.0)
        else:
            margins.append(np.inf)
        j = int(idx[b])
        piv.append(j)
        diag.append(best)
        cand[j] = False
        # new basis direction: the normalised residual of the chosen column
        # (Q spans the chosen columns, the Q factor of QR(A, r) in Sec. 2),
        # orthogonalised once more against the basis; a residual that is
        # exactly zero adds a zero column (the chosen column is already in
        # span(Q) and T_tt = 0)
        q = np.zeros(p, dtype=Q.dtype)
        if best > 0.0:
            q = R[:, b] / best
            q = q - Q @ (Q.conj().T @ q)
            nq = np.linalg.norm(q)
            q = q / nq if nq > 0.0 else np.zeros(p, dtype=Q.dtype)
        Q = np.concatenate([Q, q[:, None]], axis=1)
    if forced is not None:
        return piv, diag, margins, Q, valid  # invalid steps hold (step, best, forced, noise)
    return piv, diag, margins, Q


def strong_rrqr_criterion(M, piv, rest):
    """Gu & Eisenstat's swap criterion for a chosen column set: with
    M(:, piv) = Q R11 (thin QR, piv in order), R12 = Q^H M(:, rest) and
    gamma_j the norm of column j of the residual (I - Q Q^H) M(:, rest),
    rho_ij = |(R11^{-1} R12)_ij|^2 + (omega_i gamma_j)^2, omega_i the norm of
    row i of R11^{-1}; sqrt(rho_ij) is the factor by which swapping chosen
    column i for candidate j multiplies |det R11|.  Returns rho (k x len(rest))
    or None when R11 is singular."""
    A = M[:, piv]
    Q, R11 = np.linalg.qr(A)
    if np.any(np.abs(np.diag(R11)) == 0.0):
        return None
    B = M[:, rest]
    R12 = Q.conj().T @ B
    gam = np.linalg.norm(B - Q @ R12, axis=0)
    Ri = scipy.linalg.solve_triangular(R11, np.eye(len(piv)), lower=False)
    om = np.linalg.norm(Ri, axis=1)
    return np.abs(Ri @ R12) ** 2 + (om[:, None] * gam[None, :]) ** 2


def strong_rrqr(M, piv, candidates=None, f=2.0, max_swaps=None):
    """Strong rank-revealing QR (Gu & Eisenstat, SIAM J. Sci. Comput. 1996) as
    a refinement of a chosen column set (one of the subset-selection methods
    Sec. 3.2 names beside QRCP): while some chosen column i and candidate j
    have rho_ij > f^2 (strong_rrqr_criterion), the largest such pair is
    swapped (ties: smallest j, then smallest i), the candidate taking the
    chosen column's position.  Every swap multiplies |det R11| by more than f,
    so the loop ends; when the set has as many columns as M has rows this is
    the maximum-volume (dominant submatrix) condition.  A singular R11 is left
    as it is.  Returns (piv, number of swaps)."""
    M = np.asarray(M)
    N = M.shape[1]
    piv = list(piv)
    k = len(piv)
    cand = np.ones(N, bool) if candidates is None else np.array(candidates, bool)
    swaps = 0
    max_swaps = 4 * k + 4 if max_swaps is None else max_swaps
    while k > 0 and swaps < max_swaps:
        chosen = np.zeros(N, bool)
        chosen[piv] = True
        rest = np.flatnonzero(cand & ~chosen)
        if rest.size == 0:
            break
        rho = strong_rrqr_criterion(M, piv, rest)
        if rho is None:
            break
        best = rho.max()
        if not best > f * f:
            break
        ii, jj = np.nonzero(rho == best)
        o = np.lexsort((ii, jj))[0]
        piv[int(ii[o])] = int(rest[jj[o]])
        swaps += 1
    return piv, swaps


def strong_rrqr_margin(M, piv, candidates=None, f=2.0):
    """Relative margin of the stopping decision of a strong RRQR set: how far
    the largest rho_ij lies below f^2, (f^2 - max rho) / f^2 (negative when a
    swap is still due; inf without candidates or with a singular R11)."""
    M = np.asarray(M)
    N = M.shape[1]
    cand = np.ones(N, bool) if candidates is None else np.array(candidates, bool)
    chosen = np.zeros(N, bool)
    chosen[list(piv)] = True
    rest = np.flatnonzero(cand & ~chosen)
    if rest.size == 0 or len(piv) == 0:
        return np.inf
    rho = strong_rrqr_criterion(M, list(piv), rest)
    if rho is None:
        return np.inf
    return float((f * f - rho.max()) / (f * f))


def eps_rank(s, eps):
    """eps-rank of a descending singular value list (Sec. 2)."""
    s = np.asarray(s)
    if s.size == 0 or s[0] == 0.0:
        return 0
    return int(np.count_nonzero(s >= eps * s[0]))


def frob_rank(s, eps_loc):
    """Smallest t with sqrt(sum_{j >= t} s_j^2) <= eps_loc sqrt(sum_j s_j^2)
    for a descending singular value list s (0-based: s[t:] is discarded).
    By Eckart and Young the rank-t truncation of A then has Frobenius error
    at most eps_loc ||A||_F and every smaller rank has more."""
    s = np.asarray(s, dtype=np.float64)
    total = np.sqrt(np.sum(s * s))
    for t in range(s.size + 1):
        if np.sqrt(np.sum(s[t:] * s[t:])) <= eps_loc * total:
            return t
    return s.size


def truncated_svd(A, eps, rank=None, frob=False):
    """[U, Sigma, V, r] = SVD(A, eps) (Sec. 2): LAPACK gesdd with a gesvd
    fallback, truncated at the eps-rank, at frob_rank(s, eps) when ``frob``
    (eps is then the truncation's own Frobenius budget), or at ``rank`` when
    given (a frozen truncation rank, used to differentiate the map with its
    discrete choices held fixed).  Returns U (m x r), s (r), Vh (r x n)."""
    A = np.asarray(A)
    m, n = A.shape
    if m == 0 or n == 0:
        return (np.zeros((m, 0), A.dtype), np.zeros(0), np.zeros((0, n), A.dtype))
    try:
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
    except np.linalg.LinAlgError:
        import scipy.linalg
        U, s, Vh = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesvd")
    if rank is not None:
        r = min(int(rank), s.size)
    else:
        r = frob_rank(s, eps) if frob else eps_rank(s, eps)
    return U[:, :r], s[:r], Vh[:r]
