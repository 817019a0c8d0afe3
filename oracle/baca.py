"""ACA (Alg. 1) and BACA (Alg. 2) with LRID, LRnorm, LRnormUp, and the SVD
re-compression of Sec. 3.2 (last paragraph).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper taken here (the CUDA path takes the same ones):
* J_1 comes from the counter-based sampler in ``sampler`` (Alg. 2 line 1).
* Row exclusion (Sec. 3.2): I_k is chosen among rows not kept by earlier
  iterations (kept rows are I_j(1:d_j), Alg. 2 line 9).
* Column exclusion: J_{k+1} is chosen among columns not kept by earlier
  iterations and not in the current J_k (J_k is still unshrunk when line 6
  runs).  Columns of J_k dropped by LRID become eligible again later.
* QR(C_k^t, d) and QR(R_k, d) select at most min(d, #rows of the matrix,
  #candidates) pivots.  Fewer candidates than d: all of them are taken.
* W_k = E_{k-1}(I_k, J_k) is read out of C_k (same residual entries).
* QR(W, eps) keeps the leading pivots whose residual norm |T_tt| is at least
  eps |T_11|; d_k = 0 when T_11 = 0 (then nothing is appended and nu = 0).
* LRnorm uses the identity ||U V||_F^2 = sum_ij (U^H U)_ij conj((V V^H)_ij),
  which equals the Cholesky form of Eqs. chol/numu without forming factors.
  LRnormUp adds 2 Re sum (U^H U_k) o conj(V V_k^H) (Eq. normup; the
  conjugates make it the complex form).
* The stopping test nu < eps mu is strict, after the update (lines 12-14).
  The loop also ends when no candidate row or column remains, or after
  min(m, n) iterations (line 2).
* Complex data: transposes in QR(V^t) and Q^t are conjugate transposes.
"""
import numpy as np
import scipy.linalg

from .linalg import greedy_qrcp, truncated_svd
from .sampler import initial_columns


def lrid(C, W, R, eps):
    """LRID(C, W, R, eps) of Alg. 2 (Eqs. LRID1, LRID2).

    Returns U_k = C(:, Jbar), V_k = T^{-1} Q^H R, d_k and Jbar (positions
    into the columns of W, in pivot order)."""
    dI, dJ = W.shape
    piv, diag, _, Q = greedy_qrcp(W, min(dI, dJ), rank_tol=eps)
    dk = len(piv)
    if dk == 0:
        return C[:, :0], R[:0, :], 0, []
    T = np.triu(Q.conj().T @ W[:, piv])
    Uk = C[:, piv]
    Vk = scipy.linalg.solve_triangular(T, Q.conj().T @ R, lower=False)
    return Uk, Vk, dk, piv


def lrnorm(Uk, Vk):
    """LRnorm(U, V) = ||U V||_F (Alg. 2; Eqs. chol, numu), via the Gram identity."""
    GU = Uk.conj().T @ Uk
    GV = Vk @ Vk.conj().T
    s = np.real(np.sum(GU * GV.conj()))
    return float(np.sqrt(max(s, 0.0)))


def lrnorm_cholesky(Uk, Vk):
    """The paper's literal form: T1 = Chol(U^H U), T2 = Chol(V V^H),
    nu = ||T1 T2^H||_F (Eqs. chol, numu).  Needs full-rank Grams."""
    T1 = np.linalg.cholesky(Uk.conj().T @ Uk).conj().T
    T2 = np.linalg.cholesky(Vk @ Vk.conj().T).conj().T
    return float(np.linalg.norm(T1 @ T2.conj().T))


def lrnormup(U, V, mu, Uk, Vk, nu):
    """LRnormUp(U, V, mu, U_k, V_k, nu) = ||[U, U_k][V; V_k]||_F (Eq. normup)."""
    cross = np.real(np.sum((U.conj().T @ Uk) * (V @ Vk.conj().T).conj()))
    s = mu * mu + nu * nu + 2.0 * cross
    return float(np.sqrt(max(s, 0.0)))


def baca(gen, d, eps, seed=0, bid=0):
    """BACA (Alg. 2) on the whole matrix of ``gen`` (local indices).

    Returns a dict with U (m x r), V (r x n), rank r, and ``trace``: one
    record per iteration with the column block J (before LRID), the row
    pivots I (QRCP order, before shrinking), their margins, the next column
    block and its margins, Jbar, d_k, nu and mu."""
    m, n = gen.m, gen.n
    dt = np.dtype(gen.dtype)
    U = np.zeros((m, 0), dt)
    V = np.zeros((0, n), dt)
    mu = 0.0
    kept_rows = np.zeros(m, bool)
    kept_cols = np.zeros(n, bool)
    J = initial_columns(seed, bid, n, d)
    trace = []
    allrows, allcols = np.arange(m), np.arange(n)
    stop = "iterations"
    for _k in range(min(m, n)):
        if len(J) == 0:
            stop = "no columns"
            break
        C = gen(allrows, J) - U @ V[:, J]
        I, _, imarg, _ = greedy_qrcp(C.T, d, candidates=~kept_rows)
        if len(I) == 0:
            stop = "no rows"
            break
        R = gen(I, allcols) - U[I, :] @ V
        cand = ~kept_cols
        cand[J] = False
        Jn, _, jmarg, _ = greedy_qrcp(R, d, candidates=cand)
        W = C[I, :]
        Uk, Vk, dk, jbar = lrid(C, W, R, eps)
        nu = lrnorm(Uk, Vk) if dk else 0.0
        mu = lrnormup(U, V, mu, Uk, Vk, nu) if dk else mu
        U = np.concatenate([U, Uk], axis=1)
        V = np.concatenate([V, Vk], axis=0)
        kept_rows[I[:dk]] = True
        kept_cols[[J[p] for p in jbar]] = True
        trace.append(dict(J=list(J), I=list(I), Imarg=imarg, Jnext=list(Jn),
                          Jmarg=jmarg, jbar=list(jbar), dk=dk, nu=nu, mu=mu))
        if nu < eps * mu:
            stop = "converged"
            break
        J = Jn
    return dict(U=U, V=V, r=U.shape[1], trace=trace, stop=stop, mu=mu)


def aca(gen, eps, seed=0, bid=0):
    """Partially pivoted ACA exactly as Alg. 1 (Eqs. iik, jjk, aca_stop).

    A zero pivot u_k(i_k) = 0 (division by zero at line 5) is read as an
    empty update: nothing is appended, nu = 0, i_k and j_k stay eligible."""
    m, n = gen.m, gen.n
    dt = np.dtype(gen.dtype)
    U = np.zeros((m, 0), dt)
    V = np.zeros((0, n), dt)
    mu = 0.0
    used_i = np.zeros(m, bool)
    used_j = np.zeros(n, bool)
    j = initial_columns(seed, bid, n, 1)[0]
    piv = []
    allrows, allcols = np.arange(m), np.arange(n)
    for _k in range(min(m, n)):
        u = gen(allrows, [j])[:, 0] - U @ V[:, j]
        au = np.where(used_i, -1.0, np.abs(u))
        if au.max() < 0:
            break
        i = int(np.argmax(au))
        v = gen([i], allcols)[0] - U[i, :] @ V
        cand = ~used_j
        cand[j] = False
        av = np.where(cand, np.abs(v), -1.0)
        jn = int(np.argmax(av)) if av.max() >= 0 else None
        if u[i] == 0:
            nu = 0.0
        else:
            u = u / u[i]
            nu = float(np.linalg.norm(u) * np.linalg.norm(v))
            cross = np.real(np.sum((U.conj().T @ u) * (V @ v.conj()).conj()))
            mu = float(np.sqrt(max(mu * mu + nu * nu + 2.0 * cross, 0.0)))
            U = np.concatenate([U, u[:, None]], axis=1)
            V = np.concatenate([V, v[None, :]], axis=0)
            used_i[i] = True
            used_j[j] = True
            piv.append((i, j))
        if nu < eps * mu:
            break
        if jn is None:
            break
        j = jn
    return dict(U=U, V=V, r=U.shape[1], piv=piv, mu=mu)


def recompress(U, V, eps):
    """SVD re-compression of U V (Sec. 3.2, last paragraph):
    [Q_U, T_U] = QR(U), [Q_V, T_V] = QR(V^H), SVD(T_U T_V^H, eps) = X S Y^H;
    returns (Q_U X, s, Y^H Q_V^H)."""
    m, r = U.shape
    n = V.shape[1]
    if r == 0:
        return U[:, :0], np.zeros(0), V[:0, :]
    Qu, Tu = np.linalg.qr(U)
    Qv, Tv = np.linalg.qr(V.conj().T)
    X, s, Yh = truncated_svd(Tu @ Tv.conj().T, eps)
    return Qu @ X, s, Yh @ Qv.conj().T
