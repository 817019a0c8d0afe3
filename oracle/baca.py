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

from .linalg import greedy_qrcp, strong_rrqr, strong_rrqr_margin, truncated_svd
from .sampler import initial_columns


def lrid(C, W, R, eps):
    """LRID(C, W, R, eps) of Alg. 2 (Eqs. LRID1, LRID2).

    Returns U_k = C(:, Jbar), V_k = T^{-1} Q^H R, d_k and Jbar (positions
    into the columns of W, in pivot order).  With ``info`` the QRCP margins
    and |T_tt| are returned as a fifth element."""
    return _lrid(C, W, R, eps)[:4]


def _noise(A, absUV):
    """Absolute rounding-noise level of the norms of residual vectors
    A - U V (d-vectors): 1e-12 * sqrt(d) * max(|A|, |U| |V|), where absUV is
    the product of the entry-wise magnitudes (cancellation in U V leaves
    rounding errors proportional to it, not to |U V|)."""
    scale = max(float(np.abs(A).max(initial=0.0)), float(np.abs(absUV).max(initial=0.0)))
    return 1e-12 * np.sqrt(max(A.shape[0] if A.ndim == 1 else min(A.shape), 1)) * scale


def _lrid(C, W, R, eps, noise=0.0):
    dI, dJ = W.shape
    piv, diag, marg, Q = greedy_qrcp(W, min(dI, dJ), rank_tol=eps, abs_noise=noise)
    # the first rejected candidate (for the margin of the rank decision)
    full, fdiag, _, _ = greedy_qrcp(W, min(dI, dJ), abs_noise=noise)
    info = dict(marg=marg, diag=diag, noise=noise,
                next=(fdiag[len(piv)] if len(fdiag) > len(piv) else None))
    dk = len(piv)
    if dk == 0:
        return C[:, :0], R[:0, :], 0, [], info
    T = np.triu(Q.conj().T @ W[:, piv])
    Uk = C[:, piv]
    Vk = scipy.linalg.solve_triangular(T, Q.conj().T @ R, lower=False)
    return Uk, Vk, dk, piv, info


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


def _refine(diag, mu):
    """Whether a greedy pivot set is refined by strong RRQR: only a set whose
    smallest pivot residual norm is at least 1e-8 of the larger of the first
    one and the current mu.  Below that the chosen block is numerically
    rank-deficient or at the rounding level, where the swap criterion
    compares rounding noise and volume gains mean nothing."""
    return len(diag) > 0 and min(diag) >= 1e-8 * max(diag[0], mu)


def baca(gen, d, eps, seed=0, bid=0, srrqr_f=None):
    """BACA (Alg. 2) on the whole matrix of ``gen`` (local indices).

    Returns a dict with U (m x r), V (r x n), rank r, and ``trace``: one
    record per iteration with the column block J (before LRID), the row
    pivots I (QRCP order, before shrinking), their margins, the next column
    block and its margins, Jbar, d_k, nu and mu.

    ``srrqr_f``: select I_k and J_{k+1} by strong rank-revealing QR (Sec. 3.2
    names it among the alternatives to QRCP): the greedy QRCP sets refined by
    Gu and Eisenstat's swaps with threshold f (linalg.strong_rrqr), when the
    greedy set is numerically of full rank (_refine); each record then also
    holds the number of swaps and the stopping margins."""
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
        AJ = gen(allrows, J)
        UVJ = U @ V[:, J]
        C = AJ - UVJ
        nC = _noise(AJ, np.abs(U) @ np.abs(V[:, J]))
        I, dgI, imarg, _ = greedy_qrcp(C.T, d, candidates=~kept_rows, abs_noise=nC)
        if len(I) == 0:
            stop = "no rows"
            break
        swI = swJ = 0
        smI = smJ = np.inf
        if srrqr_f is not None and _refine(dgI, mu):
            I, swI = strong_rrqr(C.T, I, candidates=~kept_rows, f=srrqr_f)
            smI = strong_rrqr_margin(C.T, I, candidates=~kept_rows, f=srrqr_f)
        AI = gen(I, allcols)
        UVI = U[I, :] @ V
        R = AI - UVI
        cand = ~kept_cols
        cand[J] = False
        Jn, dgJ, jmarg, _ = greedy_qrcp(R, d, candidates=cand, abs_noise=_noise(AI, np.abs(U[I, :]) @ np.abs(V)))
        if srrqr_f is not None and len(Jn) and _refine(dgJ, mu):
            Jn, swJ = strong_rrqr(R, Jn, candidates=cand, f=srrqr_f)
            smJ = strong_rrqr_margin(R, Jn, candidates=cand, f=srrqr_f)
        W = C[I, :]
        Uk, Vk, dk, jbar, winfo = _lrid(C, W, R, eps, nC)
        nu = lrnorm(Uk, Vk) if dk else 0.0
        mu = lrnormup(U, V, mu, Uk, Vk, nu) if dk else mu
        U = np.concatenate([U, Uk], axis=1)
        V = np.concatenate([V, Vk], axis=0)
        kept_rows[I[:dk]] = True
        kept_cols[[J[p] for p in jbar]] = True
        trace.append(dict(J=list(J), I=list(I), Imarg=imarg, Jnext=list(Jn),
                          Jmarg=jmarg, jbar=list(jbar), dk=dk, nu=nu, mu=mu, W=winfo,
                          swaps=(swI, swJ), smarg=(smI, smJ)))
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


def recompress(U, V, eps, rank=None, frob=False):
    """SVD re-compression of U V (Sec. 3.2, last paragraph):
    [Q_U, T_U] = QR(U), [Q_V, T_V] = QR(V^H), SVD(T_U T_V^H, eps) = X S Y^H;
    returns (Q_U X, s, Y^H Q_V^H).  ``rank`` freezes the truncation rank;
    ``frob`` truncates by the Frobenius rule (linalg.frob_rank) with budget
    eps."""
    m, r = U.shape
    n = V.shape[1]
    if r == 0:
        return U[:, :0], np.zeros(0), V[:0, :]
    Qu, Tu = np.linalg.qr(U)
    Qv, Tv = np.linalg.qr(V.conj().T)
    X, s, Yh = truncated_svd(Tu @ Tv.conj().T, eps, rank, frob)
    return Qu @ X, s, Yh @ Qv.conj().T


def _srrqr_set_ok(M, forced, cand, k_expect, f, noise):
    """A forced set of a strong-RRQR run: distinct candidates, as many as the
    greedy selection takes, and no swap left above f^2 (up to rounding), or a
    matrix at the rounding level."""
    forced = list(forced)
    if len(forced) != k_expect or len(set(forced)) != len(forced) or not all(cand[j] for j in forced):
        return False
    if k_expect == 0 or float(np.abs(M).max(initial=0.0)) <= 100.0 * noise:
        return True
    return strong_rrqr_margin(M, forced, candidates=cand, f=f) >= -1e-8


def baca_replay(gen, d, eps, trace, seed=0, bid=0, stop="converged", srrqr_f=None):
    """Frozen-pivot BACA: Alg. 2 with the pivot choices I_k, J_{k+1}, Jbar,
    d_k and the iteration count taken from ``trace`` (a record of another
    run, e.g. the CUDA path).  Every forced choice is checked to be a valid
    greedy choice up to rounding noise; the arithmetic (residuals, LRID,
    norms) is the oracle's own.

    ``stop`` is the recorded reason the run ended ("converged", "no columns",
    "no rows", "iterations"); the last record's valid_stop checks it.

    Returns U, V, r and per-iteration records with the validity flags
    (valid_I, valid_J, valid_W, valid_dk, valid_stop), nu, mu and
    noise_level (W at the rounding-noise level; records after the first such
    one are not comparable with the recorded run).

    ``srrqr_f``: the recorded run selected I_k and J_{k+1} by strong RRQR with
    threshold f; a forced set is then valid when it has the greedy count of
    distinct candidates and no swap above f^2 is left (its defining
    property) rather than when it is the greedy choice."""
    m, n = gen.m, gen.n
    dt = np.dtype(gen.dtype)
    U = np.zeros((m, 0), dt)
    V = np.zeros((0, n), dt)
    mu = 0.0
    kept_rows = np.zeros(m, bool)
    kept_cols = np.zeros(n, bool)
    J = initial_columns(seed, bid, n, d)
    allrows, allcols = np.arange(m), np.arange(n)
    recs = []
    for k, t in enumerate(trace):
        rec = dict(J_ok=list(J) == list(t["J"]))
        J = list(t["J"])
        AJ = gen(allrows, J)
        UVJ = U @ V[:, J]
        C = AJ - UVJ
        nC = _noise(AJ, np.abs(U) @ np.abs(V[:, J]))
        if srrqr_f is None:
            I, _, _, _, vI = greedy_qrcp(C.T, d, candidates=~kept_rows, abs_noise=nC, forced=list(t["I"]))
            rec["valid_I"] = all(v is True for v in vI) and len(I) == len(t["I"])
        else:
            gI, dgI, _, _ = greedy_qrcp(C.T, d, candidates=~kept_rows, abs_noise=nC)
            if _refine(dgI, mu):
                I = list(t["I"])
                vI = [_srrqr_set_ok(C.T, I, ~kept_rows, len(gI), srrqr_f, nC)]
            else:
                I, _, _, _, vI = greedy_qrcp(C.T, d, candidates=~kept_rows, abs_noise=nC, forced=list(t["I"]))
            rec["valid_I"] = all(v is True for v in vI) and len(I) == len(t["I"])
        if not rec["valid_I"]:
            rec["why"] = [v for v in vI if v is not True]
            recs.append(rec)
            break
        AI = gen(I, allcols)
        UVI = U[I, :] @ V
        R = AI - UVI
        cand = ~kept_cols
        cand[J] = False
        nR = _noise(AI, np.abs(U[I, :]) @ np.abs(V))
        gJ, dgJ, _, _ = greedy_qrcp(R, d, candidates=cand, abs_noise=nR) if srrqr_f is not None else (0, 0, 0, 0)
        if k + 1 < len(trace) and srrqr_f is not None and _refine(dgJ, mu):
            rec["valid_J"] = _srrqr_set_ok(R, trace[k + 1]["J"], cand, len(gJ), srrqr_f, nR)
        elif k + 1 < len(trace):
            Jn, _, _, _, vJ = greedy_qrcp(R, d, candidates=cand, abs_noise=_noise(AI, np.abs(U[I, :]) @ np.abs(V)),
                                          forced=list(trace[k + 1]["J"]))
            # the forced block must also be as long as the greedy rule allows
            rec["valid_J"] = all(v is True for v in vJ) and len(Jn) == min(d, len(I), int(cand.sum()))
        else:
            rec["valid_J"] = True
        ncand_next = int(cand.sum())
        W = C[I, :]
        dI, dJ = W.shape
        jbar = list(t["jbar"])
        dk = t["dk"]
        piv, diag, _, Q, vW = greedy_qrcp(W, min(dI, dJ), abs_noise=nC, forced=jbar, rank_tol=eps)
        rec["valid_W"] = all(v is True for v in vW) and len(piv) == dk
        # a cross W whose largest residual column is within 100x the rounding
        # level carries no information, and a kept pivot |T_tt| within 1e4x of
        # it is rounding-dominated: LRID's relative rank rule keeps it and
        # T^-1 amplifies the noise, after which two correct implementations
        # legitimately part ways
        rec["noise_level"] = bool(len(diag) == 0 or diag[0] <= 100.0 * nC
                                  or (dk > 0 and min(diag[:dk]) <= 1e4 * nC))
        # condition number of the kept triangle: rounding in V_k = T^-1 Q^H R
        # (and so in nu, mu) is amplified by it
        rec["cond_T"] = float(diag[0] / min(diag[:dk])) if dk > 0 else 1.0
        # relative rounding level of the smallest kept pivot: the update
        # C T^-1 Q^H R inherits it (a diagnostic for comparisons, not used here)
        rec["w_noise"] = float(nC / min(diag[:dk])) if dk > 0 and min(diag[:dk]) > 0 else 0.0
        # rank rule QR(W, eps): kept pivots at or above eps |T_11|, the next one below
        nxt = greedy_qrcp(W, min(dI, dJ), abs_noise=nC)[1]
        ok = True
        if dk > 0:
            ok = all(x >= eps * diag[0] - nC for x in diag[:dk])
            if dk < len(nxt):
                ok = ok and nxt[dk] < eps * diag[0] + nC + 1e-9 * diag[0]
        else:
            ok = len(nxt) == 0 or nxt[0] <= nC
        rec["valid_dk"] = ok
        if dk > 0:
            T = np.triu(Q.conj().T @ W[:, piv])
            if np.any(np.diag(T) == 0.0):
                # a forced pivot whose residual is exactly zero in this
                # arithmetic (the recorded run saw rounding noise there): T^-1
                # of LRID does not exist here, as for ACA's zero pivot (Alg. 1
                # line 5); the record is at the rounding level and the replay
                # ends with it
                rec["noise_level"] = True
                rec["singular_T"] = True
                recs.append(rec)
                break
            Uk = C[:, piv]
            Vk = scipy.linalg.solve_triangular(T, Q.conj().T @ R, lower=False)
            nu = lrnorm(Uk, Vk)
            mu = lrnormup(U, V, mu, Uk, Vk, nu)
            U = np.concatenate([U, Uk], axis=1)
            V = np.concatenate([V, Vk], axis=0)
        else:
            nu = 0.0
        kept_rows[I[:dk]] = True
        kept_cols[[J[p] for p in jbar]] = True
        last = k + 1 == len(trace)
        # the stop decision, with slack for rounding in nu and mu
        tol = 1e-9 * mu
        converged = nu < eps * mu + tol
        if not last:
            rec["valid_stop"] = nu >= eps * mu - tol
        elif stop == "converged":
            rec["valid_stop"] = converged
        elif stop == "no columns":
            rec["valid_stop"] = ncand_next == 0
        elif stop == "no rows":
            rec["valid_stop"] = bool(kept_rows.all())
        elif stop == "iterations":
            rec["valid_stop"] = len(trace) == min(m, n)
        else:
            rec["valid_stop"] = False
        rec.update(nu=nu, mu=mu, dk=dk)
        recs.append(rec)
        if k + 1 < len(trace):
            J = list(trace[k + 1]["J"])
    return dict(U=U, V=V, r=U.shape[1], recs=recs, mu=mu)
