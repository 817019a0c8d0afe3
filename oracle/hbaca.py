"""H-BACA: leaf-level BACA followed by the hierarchical low-rank merge
(Alg. 3; Sec. 3.3, Eqs. columncomb, columnsvdmerge).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings: both index trees have L levels (n_b = 4^L leaves); a node of size
s splits into a first child of ceil(s/2) and a second of floor(s/2) ("approximately
equal sizes", Sec. 3.3).  Each merge is the literal SVD(., eps) of Sec. 2
applied to the stacked factor (LAPACK gesdd), then the product with the
other stacked factor.

Optional Frobenius truncation (trunc="frob"): the accuracy the paper reports
is the relative Frobenius error (Sec. 5.2), and a block passes through 2L + 1
truncations (its leaf re-compression, then a horizontal and a vertical merge
per level); each of them keeps the fewest singular triplets whose discarded
tail is at most eps_loc = eps / sqrt(2L + 1) of that block's Frobenius norm,
so the budgets add up to eps in quadrature.  BACA's own stopping test keeps
eps.
"""
import numpy as np

from .baca import baca, baca_replay, recompress
from .generators import Window
from .linalg import truncated_svd
from .sampler import block_id


def tree_levels(n, L):
    """Nodes of an L-level binary tree on [0, n): list indexed by level l
    (0 = leaves, L = root) of (start, size) pairs, left to right."""
    levels = [[(0, n)]]
    for _ in range(L):
        nxt = []
        for (s, sz) in levels[0]:
            a = (sz + 1) // 2
            nxt.append((s, a))
            nxt.append((s + a, sz - a))
        levels.insert(0, nxt)
    return levels


def horizontal_merge(U1, s1, V1, U2, s2, V2, eps, rank=None, frob=False):
    """Eqs. columncomb, columnsvdmerge: U_bar = [U1 S1, U2 S2],
    V_bar = diag(V1, V2); [U, S, V'] = SVD(U_bar, eps); V = V' V_bar."""
    Ub = np.concatenate([U1 * s1[None, :], U2 * s2[None, :]], axis=1)
    r1, r2 = V1.shape[0], V2.shape[0]
    Vb = np.zeros((r1 + r2, V1.shape[1] + V2.shape[1]), np.result_type(V1, V2))
    Vb[:r1, :V1.shape[1]] = V1
    Vb[r1:, V1.shape[1]:] = V2
    U, s, Vp = truncated_svd(Ub, eps, rank, frob)
    return U, s, Vp @ Vb


def vertical_merge(U1, s1, V1, U2, s2, V2, eps, rank=None, frob=False):
    """Alg. 3 lines 17-20: U_bar = diag(U1, U2), V_bar = [S1 V1; S2 V2];
    [U', S, V] = SVD(V_bar, eps); U = U_bar U'."""
    r1, r2 = U1.shape[1], U2.shape[1]
    Ub = np.zeros((U1.shape[0] + U2.shape[0], r1 + r2), np.result_type(U1, U2))
    Ub[:U1.shape[0], :r1] = U1
    Ub[U1.shape[0]:, r1:] = U2
    Vb = np.concatenate([s1[:, None] * V1, s2[:, None] * V2], axis=0)
    Up, s, V = truncated_svd(Vb, eps, rank, frob)
    return Ub @ Up, s, V


def frob_budget(eps, L):
    """Frobenius budget of one truncation of an L-level H-BACA: the 2L + 1
    truncations a block passes through share eps in quadrature."""
    return eps / np.sqrt(2.0 * L + 1.0)


def hbaca(gen, L, d, eps, seed=0, batch_index=0, keep_leaves=False, forced=None, ranks=None, trunc="sigma"):
    """H-BACA(A, n_b = 4^L, d, eps) of Alg. 3.  Returns a dict with U, s, V,
    rank r, the leaf BACA results (if ``keep_leaves``), the leaf ranks before
    and after re-compression, and the merge ranks per level.  ``forced``
    maps a leaf index a * 2^L + b to a pivot record {"trace": [...], "stop":
    reason}; those leaves are run by
    the frozen-pivot replay (baca_replay) instead of the greedy choices.
    ``ranks`` freezes truncation ranks: it maps ("full", 0, a, b) (leaf
    re-compression), ("half", l, a, b) and ("full", l, a, b) (merges) to a
    rank; the result's "ranks" entry lists every truncation rank taken, in the
    same keys, so that one run's choices can be frozen in another.
    ``trunc``: "sigma" (the eps-rank of Sec. 2) or "frob" (each truncation
    keeps the fewest triplets whose tail is at most frob_budget(eps, L) of the
    block's Frobenius norm)."""
    if trunc not in ("sigma", "frob"):
        raise ValueError("trunc must be 'sigma' or 'frob'")
    frob = trunc == "frob"
    et = frob_budget(eps, L) if frob else eps
    taken = {}

    def rk(key):
        return None if ranks is None else ranks.get(key)
    rows = tree_levels(gen.m, L)
    cols = tree_levels(gen.n, L)
    blocks = {}
    leaf_info = {}
    for a, (r0, mr) in enumerate(rows[0]):
        for b, (c0, nc) in enumerate(cols[0]):
            w = Window(gen, r0, mr, c0, nc)
            leaf = a * len(cols[0]) + b
            if forced is not None and leaf in forced:
                fr = forced[leaf]
                res = baca_replay(w, d, eps, fr["trace"], seed=seed, bid=block_id(batch_index, a, b),
                                  stop=fr.get("stop", "converged"))
                res["trace"] = res["recs"]
                res["stop"] = "replayed"
            else:
                res = baca(w, d, eps, seed=seed, bid=block_id(batch_index, a, b))
            U, s, V = recompress(res["U"], res["V"], et, rk(("full", 0, a, b)), frob)
            taken[("full", 0, a, b)] = len(s)
            blocks[(a, b)] = (U, s, V)
            info = dict(r_baca=res["r"], r=len(s), iters=len(res["trace"]), stop=res["stop"])
            if keep_leaves:
                info["baca"] = res
            leaf_info[(a, b)] = info
    merge_ranks = []
    stages = [("full", 0, dict(blocks))] if keep_leaves else []
    for l in range(1, L + 1):
        half = {}
        for a in range(len(rows[l - 1])):
            for b in range(len(cols[l])):
                U1, s1, V1 = blocks[(a, 2 * b)]
                U2, s2, V2 = blocks[(a, 2 * b + 1)]
                half[(a, b)] = horizontal_merge(U1, s1, V1, U2, s2, V2, et, rk(("half", l, a, b)), frob)
                taken[("half", l, a, b)] = len(half[(a, b)][1])
        full = {}
        for a in range(len(rows[l])):
            for b in range(len(cols[l])):
                U1, s1, V1 = half[(2 * a, b)]
                U2, s2, V2 = half[(2 * a + 1, b)]
                full[(a, b)] = vertical_merge(U1, s1, V1, U2, s2, V2, et, rk(("full", l, a, b)), frob)
                taken[("full", l, a, b)] = len(full[(a, b)][1])
        merge_ranks.append(dict(half={k: len(v[1]) for k, v in half.items()},
                                full={k: len(v[1]) for k, v in full.items()}))
        if keep_leaves:
            stages.append(("half", l, half))
            stages.append(("full", l, full))
        blocks = full
    U, s, V = blocks[(0, 0)]
    return dict(U=U, s=s, V=V, r=len(s), leaves=leaf_info, merges=merge_ranks, stages=stages, ranks=taken)
