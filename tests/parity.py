"""Comparison of GPU leaf records with the oracle's, following the parity
rule: pivot sequences and ranks must be identical while every decision is
unique by a relative margin of 1e-9; after the first sub-margin decision a
leaf is only compared through ranks (+-2) and errors."""
import numpy as np

MARGIN = 1e-9


def _prefix_ok(margins, thr=MARGIN):
    """Number of leading decisions with a margin above thr."""
    n = 0
    for m in margins:
        if not (m > thr):
            break
        n += 1
    return n


def compare_leaf(o, g, eps):
    """o: oracle baca() dict, g: binding.read_leaf_trace() dict.
    Returns (iterations compared, diverged flag).

    A decision counts as unique when its margin exceeds 1e-9, raised to
    1e-13 mu_j / nu_j for the largest ratio of the iterations before it: the
    residual A - U V is formed with cancellation of that size (the update of
    iteration j is nu_j against an accumulated approximation of norm mu_j),
    so two correct runs' residuals differ by about eps_mach mu / nu
    relative."""
    ot, gt = o["trace"], g["trace"]
    amp = 1.0
    for k in range(min(len(ot), len(gt))):
        a, b = ot[k], gt[k]
        assert a["J"] == b["J"], ("J", k, a["J"], b["J"])
        thr = max(MARGIN, 1e-13 * amp)
        nI = _prefix_ok(a["Imarg"], thr)
        assert a["I"][:nI] == b["I"][:nI], ("I", k, a["I"], b["I"])
        if nI < len(a["I"]):
            return k, True
        w = a["W"]
        # a cross at the rounding level, or a kept pivot within 1e4 of it: the
        # LRID triangle amplifies rounding noise and the two runs' updates
        # (nu, mu, later pivots) legitimately part ways from here on
        nz = w.get("noise", 0.0)
        if w["diag"] and (w["diag"][0] <= 100.0 * nz or (a["dk"] > 0 and min(w["diag"][:a["dk"]]) <= 1e4 * nz)):
            return k, True
        nW = _prefix_ok(w["marg"], thr)
        assert a["jbar"][:nW] == b["jbar"][:nW], ("jbar", k, a["jbar"], b["jbar"])
        if nW < len(a["jbar"]):
            return k, True
        # the eps-rank decision of QR(W, eps) is unique unless a |T_tt| sits at eps |T_11|
        d0 = w["diag"][0] if w["diag"] else 0.0
        tol = max(1e-6 * eps * d0, w.get("noise", 0.0))
        near = [abs(t - eps * d0) <= tol for t in w["diag"][1:]] if d0 else []
        if w["next"] is not None and d0:
            near.append(abs(w["next"] - eps * d0) <= tol)
        if any(near):
            return k, True
        assert a["dk"] == b["dk"], ("dk", k, a["dk"], b["dk"])
        # nu, mu are norms of the same low-rank blocks
        assert abs(a["mu"] - b["mu"]) <= 1e-9 * max(a["mu"], 1e-300), ("mu", k, a["mu"], b["mu"])
        assert abs(a["nu"] - b["nu"]) <= 1e-9 * max(a["mu"], 1e-300), ("nu", k, a["nu"], b["nu"])
        nJ = _prefix_ok(a["Jmarg"], thr)
        if k + 1 < len(ot) and k + 1 < len(gt):
            assert ot[k + 1]["J"][:nJ] == gt[k + 1]["J"][:nJ], ("Jnext", k)
        if nJ < len(a["Jnext"]):
            return k + 1, True
        if a["nu"] > 0.0:
            amp = max(amp, a["mu"] / a["nu"])
    assert len(ot) == len(gt), ("iterations", len(ot), len(gt))
    assert o["r"] == g["rank_baca"], ("rank", o["r"], g["rank_baca"])
    return len(ot), False


def dense_rel_error(A, U, s, V):
    E = A - (U * s[None, :]) @ V
    return float(np.linalg.norm(E) / np.linalg.norm(A))


def check_leaf_replay(ogen_leaf, g, d, eps, seed, bid, rounding_sensitive=False, srrqr_f=None):
    """Replay the GPU's pivot record through the oracle (frozen pivots): every
    GPU choice must be a valid greedy choice up to rounding, and the norms and
    ranks must agree.  Returns the replay result.

    rounding_sensitive: the input is one on which the method amplifies
    rounding (the coherent sparse product, see
    test_oracle_pins.test_coherent_case_is_rounding_sensitive).  There a
    forced choice that is not greedy in the oracle's arithmetic only ends the
    comparison when the competing residual norms are at the rounding level of
    the leaf (below 1e-12 times the largest mu the leaf reached): the two runs'
    residuals have parted by the amplified rounding of earlier iterations,
    which the local noise estimate of one cross does not see.

    srrqr_f: the run refined its pivot sets by strong RRQR with this
    threshold; a forced set is then valid when no swap above f^2 is left."""
    from oracle import baca as ob
    rep = ob.baca_replay(ogen_leaf, d, eps, g["trace"], seed=seed, bid=bid, stop=g["stop"], srrqr_f=srrqr_f)
    if rounding_sensitive and rep["recs"]:
        last = rep["recs"][-1]
        scale = max([r.get("mu", 0.0) for r in rep["recs"]] + [0.0])
        why = last.get("why") or []
        if not last.get("valid_I", True) and why and all(
                isinstance(w, tuple) and w[1] <= 1e-12 * scale for w in why):
            last["noise_level"] = True
            last["valid_I"] = True
            last.setdefault("valid_J", True)
            last.setdefault("valid_W", True)
            last.setdefault("valid_dk", True)
    noisy = [k for k, r in enumerate(rep["recs"]) if r.get("noise_level")]
    limit = noisy[0] + 1 if noisy else len(g["trace"])
    assert len(rep["recs"]) >= limit, ("replay stopped", len(rep["recs"]), len(g["trace"]), rep["recs"][-1])
    rep["comparable"] = True
    cond = 1.0
    for k, (r, t) in enumerate(zip(rep["recs"], g["trace"])):
        for key in ("J_ok", "valid_I", "valid_J", "valid_W", "valid_dk"):
            assert r[key], (key, k, g["stop"], r)
        if r.get("noise_level"):
            # this iteration's update is rounding-dominated: nu, mu and what
            # follows are not comparable between two correct runs
            rep["comparable"] = False
            rep["compared_iters"] = k
            break
        assert r["valid_stop"], ("valid_stop", k, g["stop"], r)
        # rounding in nu, mu grows with the conditioning of the LRID triangles so far
        cond = max(cond, r.get("cond_T", 1.0))
        tol = max(1e-9, 1e-13 * cond) * max(r["mu"], 1e-300)
        assert abs(r["mu"] - t["mu"]) <= tol, ("mu", k, r["mu"], t["mu"], cond)
        assert abs(r["nu"] - t["nu"]) <= tol, ("nu", k, r["nu"], t["nu"], cond)
    assert rep["r"] == g["rank_baca"] or not rep["comparable"]
    return rep


def near_threshold(s, eps, rel=1e-6):
    """True when an eps-rank decision on singular values s is ambiguous."""
    s = np.asarray(s)
    if s.size == 0 or s[0] == 0:
        return False
    return bool(np.any(np.abs(s / s[0] - eps) <= rel * eps))


def stable_prefix(recs, gtrace):
    """Number of leading iterations of a leaf before its first rounding-level
    cross (frozen-pivot replay records) or its first kept pivot within 1e8 of
    the rounding level (the update C T^-1 Q^H R then carries a relative
    rounding error above 1e-8), the BACA rank they add, and the largest
    relative rounding level of their kept pivots."""
    k0 = next((k for k, r in enumerate(recs) if r.get("noise_level") or r.get("w_noise", 0.0) > 1e-8), len(recs))
    k0 = min(k0, len(gtrace))
    amp = max([0.0] + [r.get("w_noise", 0.0) for r in recs[:k0]])
    return k0, sum(t["dk"] for t in gtrace[:k0]), amp
