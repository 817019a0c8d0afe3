"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(not against itself).  CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import apply as oapply
from oracle import baca as ob
from oracle import generators as og
from oracle import hbaca as oh
from oracle import linalg as ol
from oracle import sampler as osamp
from paper_1901_06101_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- sampler
def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            seed, vals = line.split(":")
            want = [int(v) for v in vals.split()]
            assert osamp.splitmix64_outputs(int(seed), len(want)) == want


def test_initial_columns_distinct_and_uniform():
    for n, d in [(1, 8), (5, 8), (500, 8), (1563, 32)]:
        J = osamp.initial_columns(7, 3, n, d)
        assert len(J) == min(n, d) and len(set(J)) == len(J)
        assert all(0 <= j < n for j in J)
    # first element uniform over [0, 10): chi-square over many streams
    counts = np.zeros(10)
    for b in range(5000):
        counts[osamp.initial_columns(11, b, 10, 3)[0]] += 1
    chi2 = ((counts - 500.0) ** 2 / 500.0).sum()
    assert chi2 < 30.0  # 9 dof, p ~ 4e-4


# ---------------------------------------------------------------- generators
def test_generator_closed_forms():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    y = np.array([[0.0, 2.0, 0.0]])
    g = og.Gaussian(x, y, 2.0)
    np.testing.assert_allclose(g([0, 1], [0])[:, 0], [np.exp(-4.0 / 8.0), np.exp(-5.0 / 8.0)], rtol=1e-15)
    hz = og.Helmholtz(x, y, np.pi)
    np.testing.assert_allclose(hz([0], [0])[0, 0], np.exp(2j * np.pi) / 2.0, rtol=1e-14)
    np.testing.assert_allclose(hz([1], [0])[0, 0], np.exp(1j * np.pi * np.sqrt(5.0)) / np.sqrt(5.0), rtol=1e-14)


def test_sparse_product_entries_by_intersection():
    sp = inputs.sparse_product(seed=5, m=300, n=280, K=7, density=0.05)
    g = og.SparseProduct(sp.dense_P(), sp.dense_Q(), sp.P2, sp.Q2)
    rng = np.random.default_rng(0)
    for _ in range(50):
        i, j = int(rng.integers(300)), int(rng.integers(280))
        # brute force: walk row i of P (CSR) and column j of Q (CSC)
        acc = 0.0
        ps, pe = sp.p_rowptr[i], sp.p_rowptr[i + 1]
        qs, qe = sp.q_colptr[j], sp.q_colptr[j + 1]
        for a in range(ps, pe):
            for b in range(qs, qe):
                if sp.p_colidx[a] == sp.q_rowidx[b]:
                    acc += sp.p_val[a] * sp.q_val[b]
        acc += sum(sp.P2[i, t] * sp.Q2[t, j] for t in range(sp.P2.shape[1]))
        assert abs(g([i], [j])[0, 0] - acc) <= 1e-14 * (1 + abs(acc))
    # exact density: each column of P / row of Q has exactly 5% nonzeros
    assert np.all((sp.dense_P() != 0).sum(axis=0) == 15)
    assert np.all((sp.dense_Q() != 0).sum(axis=1) == 14)


def test_polynomial_generator_closed_form_and_rank():
    x = np.array([[1.0, 2.0], [0.0, -1.0]])
    y = np.array([[3.0, 0.5], [1.0, 1.0]])
    g = og.Polynomial(x, y, 0.5)
    want = np.array([[(3.0 + 1.0 + 0.5) ** 2, (1.0 + 2.0 + 0.5) ** 2],
                     [(0.0 - 0.5 + 0.5) ** 2, (0.0 - 1.0 + 0.5) ** 2]])
    np.testing.assert_allclose(g([0, 1], [0, 1]), want, rtol=1e-15)
    # (x^t y + h)^2 = h^2 + 2 h x^t y + (x^t y)^2: rank 1 + dim + dim (dim + 1) / 2
    xs, ys = inputs.polynomial_pair(seed=1, m=80, n=70, dim=5)
    A = og.Polynomial(xs, ys, 0.3)(np.arange(80), np.arange(70))
    sv = np.linalg.svd(A, compute_uv=False)
    assert ol.eps_rank(sv, 1e-12) == 1 + 5 + 15


def test_hankel2d_generator_published_values():
    """H0^(2) = J0 - i Y0 at the first zeros of J0 and Y0 (Abramowitz &
    Stegun, Table 9.5: j_01 = 2.404825557695773, y_01 = 0.8935769662791675),
    the small-argument form Y0(z) ~ (2/pi)(ln(z/2) + gamma), the large-argument
    amplitude sqrt(2/(pi z)), and the distance r = 5 of a 3-4-5 triangle."""
    def H(z):
        return og.Hankel2D(np.zeros((1, 2)), np.array([[z, 0.0]]), 1.0)([0], [0])[0, 0]
    assert abs(H(2.404825557695773).real) < 1e-15
    assert abs(H(0.8935769662791675).imag) < 1e-15
    z = 1e-8
    gamma = 0.5772156649015329
    assert abs(H(z) - (1.0 - 1j * (2 / np.pi) * (np.log(z / 2) + gamma))) < 1e-13
    for z in (1e3, 1e4):
        assert abs(abs(H(z)) * np.sqrt(np.pi * z / 2) - 1.0) < 1e-3 / z
    g = og.Hankel2D(np.array([[0.0, 0.0]]), np.array([[3.0, 4.0]]), 2.0)
    assert g([0], [0])[0, 0] == H(10.0)


def test_strips_geometry():
    x, y, k = inputs.strips_pair(300)
    assert np.allclose(x[:, 1], 0.0) and np.allclose(y[:, 1], 1.0)
    assert np.allclose(np.diff(x[:, 0]), 1 / 300) and abs(x[0, 0] - 0.5 / 300) < 1e-15
    assert abs(2 * np.pi / k - 15 / 300 * 1.0) < 1e-15  # 15 points per wavelength on a strip of length 1


# ---------------------------------------------------------------- QRCP
def _separated(rng, p, N, cplx=False):
    M = rng.standard_normal((p, N)) * np.geomspace(1, 1e-3, N)[rng.permutation(N)]
    if cplx:
        M = M + 1j * rng.standard_normal((p, N)) * 0.5
    return M


@pytest.mark.parametrize("cplx", [False, True])
def test_greedy_qrcp_matches_lapack_geqp3(cplx):
    rng = np.random.default_rng(1)
    for trial in range(5):
        M = _separated(rng, 12, 40, cplx)
        piv, diag, marg, Q = ol.greedy_qrcp(M, 12)
        _, R, P = scipy.linalg.qr(M, pivoting=True, mode="economic")
        k = 0
        while k < len(piv) and marg[k] > 1e-6:
            k += 1
        assert k >= 3
        assert piv[:k] == list(P[:k])
        np.testing.assert_allclose(diag[:k], np.abs(np.diag(R))[:k], rtol=1e-10)
        np.testing.assert_allclose(Q.conj().T @ Q, np.eye(len(piv)), atol=1e-13)
        T = Q.conj().T @ M[:, piv]
        assert np.abs(np.tril(T, -1)).max() < 1e-12 * np.abs(M).max()


def test_greedy_qrcp_second_pivot_maximises_area():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((5, 30))
    piv, _, _, _ = ol.greedy_qrcp(M, 2)
    assert piv[0] == int(np.argmax(np.linalg.norm(M, axis=0)))
    areas = [abs(np.linalg.det(M[:, [piv[0], j]].T @ M[:, [piv[0], j]])) if j != piv[0] else -1
             for j in range(30)]
    assert piv[1] == int(np.argmax(areas))


def test_greedy_qrcp_candidates_and_rank_tol():
    rng = np.random.default_rng(3)
    U, V = inputs.lowrank(4, 10, 25, 3)
    M = U @ V
    cand = np.ones(25, bool)
    cand[:5] = False
    piv, diag, _, _ = ol.greedy_qrcp(M, 10, candidates=cand)
    assert all(p >= 5 for p in piv) and len(piv) == 10
    piv, diag, _, _ = ol.greedy_qrcp(M, 10, rank_tol=1e-8)
    assert len(piv) == 3
    piv, _, _, _ = ol.greedy_qrcp(np.zeros((4, 6)), 4, rank_tol=1e-8)
    assert piv == []


def test_greedy_qrcp_basis_spans_the_chosen_columns():
    """Q is the orthonormal factor of the chosen columns (QR(A, r), Sec. 2):
    M(:, piv) = Q T with T upper triangular and Q^H Q = I, also past the
    numerical rank, where the chosen residuals are at the rounding level but
    not zero (a rank-3 matrix, 6 pivots)."""
    U, V = inputs.lowrank(9, 8, 30, 3)
    M = U @ V
    piv, diag, marg, Q = ol.greedy_qrcp(M, 6)
    assert len(piv) == 6
    assert min(diag[3:]) > 0.0 and max(diag[3:]) < 1e-12 * diag[0]
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(6), atol=1e-12)
    T = Q.conj().T @ M[:, piv]
    assert np.abs(np.tril(T, -1)).max() < 1e-12 * np.abs(M).max()
    np.testing.assert_allclose(np.abs(np.diag(T)), diag, rtol=1e-6, atol=1e-14 * diag[0])
    np.testing.assert_allclose(Q @ T, M[:, piv], atol=1e-13 * np.abs(M).max())
    # an exactly zero column adds a zero direction (T_tt = 0)
    Z = np.zeros((4, 5))
    Z[:, 0] = [1.0, 2.0, 0.0, 0.0]
    piv, diag, _, Q = ol.greedy_qrcp(Z, 3)
    assert piv[0] == 0 and diag[1] == 0.0 and np.all(Q[:, 1:] == 0.0)


def _vol(M, piv):
    """|det R11| of the chosen columns, from their singular values."""
    return float(np.prod(np.linalg.svd(M[:, list(piv)], compute_uv=False)))


@pytest.mark.parametrize("p,k", [(6, 6), (9, 5)])
def test_strong_rrqr_criterion_is_the_volume_ratio_of_a_swap(p, k):
    """sqrt(rho_ij) equals |det R11| after swapping chosen column i for
    candidate j over |det R11| before (Gu & Eisenstat's Lemma), checked by
    forming every swapped set; with p > k the residual norms gamma_j enter."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((p, 20)) + 1j * rng.standard_normal((p, 20))
    piv = [3, 7, 11, 0, 15, 2][:k]
    rest = [j for j in range(20) if j not in piv]
    rho = ol.strong_rrqr_criterion(M, piv, rest)
    v0 = _vol(M, piv)
    for i in range(k):
        for jj, j in enumerate(rest):
            sw = list(piv)
            sw[i] = j
            assert abs(np.sqrt(rho[i, jj]) - _vol(M, sw) / v0) <= 1e-10 * (1 + _vol(M, sw) / v0)


def test_strong_rrqr_ends_at_a_local_volume_maximum():
    """After the refinement no single swap raises the volume by more than f
    (brute force over every swap), every swap raised it by more than f, and
    the volume is at least the greedy QRCP set's."""
    rng = np.random.default_rng(6)
    for trial in range(20):
        M = rng.standard_normal((4, 25)) @ np.diag(rng.uniform(0.3, 1.5, 25))
        g, _, _, _ = ol.greedy_qrcp(M, 4)
        for f in (1.0, 1.2):
            piv, sw = ol.strong_rrqr(M, g, f=f)
            v = _vol(M, piv)
            assert v >= _vol(M, g) * f ** sw * (1 - 1e-12)
            for i in range(4):
                for j in range(25):
                    if j in piv:
                        continue
                    t = list(piv)
                    t[i] = j
                    assert _vol(M, t) <= f * v * (1 + 1e-10)


def test_eps_rank_definition():
    assert ol.eps_rank([1.0, 0.5, 1e-7], 1e-6) == 2
    assert ol.eps_rank([2.0, 2e-6, 1e-7], 1e-6) == 2  # Sigma_{k+1} < eps Sigma_1 is strict
    assert ol.eps_rank([100.0, 1e-3, 1e-5], 1e-6) == 2  # relative to Sigma_1
    assert ol.eps_rank([0.0, 0.0], 1e-6) == 0
    assert ol.eps_rank([], 1e-6) == 0


def test_frob_rank_definition():
    """Frobenius reading of a truncation (Sec. 5.2 measures the relative
    Frobenius error): the fewest kept values whose discarded tail is at most
    eps_loc of the whole.  s = (1, 0.1, 0.01, 0.001): ||s|| = 1.0050378,
    tails from t = 1: 0.1005038, 0.0100499, 0.001, 0."""
    s = [1.0, 0.1, 0.01, 0.001]
    assert ol.frob_rank(s, 1e-4) == 4   # 1.005e-4 < 0.001
    assert ol.frob_rank(s, 5e-3) == 3   # 0.001 <= 5.025e-3 < 0.01005
    assert ol.frob_rank(s, 0.02) == 2   # 0.01005 <= 0.0201 < 0.1005
    assert ol.frob_rank(s, 0.5) == 1
    assert ol.frob_rank(s, 1.0) == 0
    assert ol.frob_rank([3.0, 4.0], 0.8) == 1  # tail 4 <= 0.8 * 5, equality kept
    assert ol.frob_rank([0.0, 0.0], 1e-6) == 0
    assert ol.frob_rank([], 1e-6) == 0


@pytest.mark.parametrize("eps_loc", [1e-1, 1e-3, 1e-7])
def test_frob_truncation_is_eckart_young_minimal(eps_loc):
    """truncated_svd(frob=True) keeps t triplets with ||A - A_t||_F <= eps_loc
    ||A||_F formed directly from A, while the best rank t - 1 approximation
    (from an independent gesvd) misses it."""
    rng = np.random.default_rng(11)
    m, n = 90, 70
    Q1, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q1 * np.logspace(0, -12, n)[None, :]) @ Q2.T
    U, s, Vh = ol.truncated_svd(A, eps_loc, frob=True)
    t = len(s)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - (U * s) @ Vh) <= eps_loc * nA * (1 + 1e-12)
    assert t >= 1
    Ug, sg, Vg = scipy.linalg.svd(A, lapack_driver="gesvd", full_matrices=False)
    prev = A - (Ug[:, :t - 1] * sg[:t - 1]) @ Vg[:t - 1]
    assert np.linalg.norm(prev) > eps_loc * nA


def _frob_rule_holds(M, t, budget, slack=1e-9):
    """t is the fewest singular values of M (dense SVD) whose discarded tail
    is at most budget ||M||_F (decisions within slack of the threshold
    accept either side)."""
    sv = np.linalg.svd(M, compute_uv=False)
    nM = np.linalg.norm(sv)
    tail = lambda k: np.linalg.norm(sv[k:])
    ok_t = tail(t) <= budget * nM * (1 + slack)
    minimal = t == 0 or tail(t - 1) > budget * nM * (1 - slack)
    return ok_t and minimal


def test_hbaca_frob_truncations_follow_the_budget():
    """trunc="frob" with L = 1: each leaf re-compression and each horizontal
    merge keeps the fewest triplets whose tail is at most eps / sqrt(3) of the
    block's Frobenius norm (2L + 1 = 3 truncations per block), checked on the
    dense blocks (the leaf's BACA product, the two re-compressed neighbours
    side by side) with numpy's SVD; the final error meets eps."""
    x, y = inputs.gaussian_pair(seed=3, m=240, n=220)
    g = og.Gaussian(x, y, 0.8)
    eps, L = 1e-5, 1
    res = oh.hbaca(g, L, 8, eps, seed=0, keep_leaves=True, trunc="frob")
    budget = eps / np.sqrt(3.0)
    leaves = dict(res["stages"][0][2])
    for (a, b), info in res["leaves"].items():
        bac = info["baca"]
        assert _frob_rule_holds(bac["U"] @ bac["V"], info["r"], budget), ("leaf", a, b)
    half = dict(res["stages"][1][2])
    for (a, b), (U, s, V) in half.items():
        U1, s1, V1 = leaves[(a, 2 * b)]
        U2, s2, V2 = leaves[(a, 2 * b + 1)]
        M = np.concatenate([(U1 * s1) @ V1, (U2 * s2) @ V2], axis=1)
        assert _frob_rule_holds(M, len(s), budget), ("half", a, b)
    A = g(np.arange(g.m), np.arange(g.n))
    err = np.linalg.norm(A - (res["U"] * res["s"]) @ res["V"]) / np.linalg.norm(A)
    assert err <= eps


def test_hbaca_frob_nb1_is_baca_plus_frob_recompression():
    """With n_b = 1 the budget is eps itself (2L + 1 = 1)."""
    g = _gauss_small()
    h = oh.hbaca(g, 0, 8, 1e-6, seed=4, trunc="frob")
    b = ob.baca(g, 8, 1e-6, seed=4, bid=osamp.block_id(0, 0, 0))
    U, s, V = ob.recompress(b["U"], b["V"], 1e-6, frob=True)
    np.testing.assert_allclose(h["s"], s, rtol=1e-12)
    assert _frob_rule_holds(b["U"] @ b["V"], len(s), 1e-6)


# ---------------------------------------------------------------- LRID / norms
@pytest.mark.parametrize("cplx", [False, True])
def test_lrid_is_interpolative_decomposition(cplx):
    rng = np.random.default_rng(4)
    m, n, d = 40, 35, 6
    A = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    I = list(rng.choice(m, d, replace=False))
    J = list(rng.choice(n, d, replace=False))
    C, R, W = A[:, J], A[I, :], A[np.ix_(I, J)]
    Uk, Vk, dk, jbar = ob.lrid(C, W, R, 1e-12)
    assert dk == d and sorted(jbar) == list(range(d))
    # full-rank W: U_k V_k = C W^{-1} R (the ID / CUR form, Sec. 3.2)
    np.testing.assert_allclose(Uk @ Vk, C @ np.linalg.solve(W, R), rtol=1e-9, atol=1e-10)
    # cross property: residual vanishes on the selected rows and columns
    E = A - Uk @ Vk
    assert np.abs(E[:, J]).max() < 1e-10 and np.abs(E[I, :]).max() < 1e-10


def test_lrid_rank_deficient_keeps_columns_exact():
    rng = np.random.default_rng(5)
    U0, V0 = inputs.lowrank(6, 30, 30, 3)
    A = U0 @ V0
    I = list(range(8))
    J = list(range(8))
    Uk, Vk, dk, jbar = ob.lrid(A[:, J], A[np.ix_(I, J)], A[I, :], 1e-10)
    assert dk == 3
    E = A - Uk @ Vk
    kept = [J[p] for p in jbar]
    assert np.abs(E[:, kept]).max() < 1e-10 * np.abs(A).max()
    # the rank-3 matrix is reproduced exactly by the rank-3 ID
    assert np.abs(E).max() < 1e-9 * np.abs(A).max()


@pytest.mark.parametrize("cplx", [False, True])
def test_lrnorm_and_update_identities(cplx):
    rng = np.random.default_rng(6)
    def mat(a, b):
        M = rng.standard_normal((a, b))
        return M + 1j * rng.standard_normal((a, b)) if cplx else M
    U, V, Uk, Vk = mat(30, 7), mat(7, 25), mat(30, 4), mat(4, 25)
    nu = ob.lrnorm(Uk, Vk)
    assert abs(nu - np.linalg.norm(Uk @ Vk)) < 1e-12 * nu
    assert abs(nu - ob.lrnorm_cholesky(Uk, Vk)) < 1e-12 * nu  # Eqs. chol, numu
    mu = np.linalg.norm(U @ V)
    mu2 = ob.lrnormup(U, V, mu, Uk, Vk, nu)
    want = np.linalg.norm(np.concatenate([U, Uk], 1) @ np.concatenate([V, Vk], 0))
    assert abs(mu2 - want) < 1e-12 * want


# ---------------------------------------------------------------- ACA / BACA
def _gauss_small(m=120, n=110, seed=8, h=0.6):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (m, 3))
    y = rng.uniform(0, 1, (n, 3)) + np.array([1.5, 0, 0])
    return og.Gaussian(x, y, h)


@pytest.mark.parametrize("gen", ["gauss", "lowrank"])
def test_baca_d1_is_aca(gen):
    """Sec. 3.2: BACA with d = 1 reduces to ACA (same pivots, same U V)."""
    g = _gauss_small() if gen == "gauss" else og.LowRank(*inputs.lowrank(9, 80, 70, 6))
    a = ob.aca(g, 1e-8, seed=3, bid=0)
    b = ob.baca(g, 1, 1e-8, seed=3, bid=0)
    # compare while the pivots are above rounding noise (nu/mu > 1e-12)
    n_ok = sum(1 for t in b["trace"] if t["dk"] == 1 and t["nu"] > 1e-12 * t["mu"])
    bp = [(t["I"][0], t["J"][0]) for t in b["trace"] if t["dk"] == 1]
    assert n_ok >= 5
    assert a["piv"][:n_ok] == bp[:n_ok]
    A = g(np.arange(g.m), np.arange(g.n))
    np.testing.assert_allclose(a["U"] @ a["V"], b["U"] @ b["V"], rtol=0, atol=1e-12 * np.abs(A).max())


def test_baca_full_block_is_qrcp_id():
    """Sec. 3.2: with d = min(m, n) BACA is the QRCP-based ID; its columns are
    LAPACK geqp3's pivots and its rank the QRCP eps-rank."""
    rng = np.random.default_rng(10)
    m = n = 40
    U0 = rng.standard_normal((m, 12)) * np.geomspace(1, 1e-9, 12)
    A = U0 @ rng.standard_normal((12, n))
    g = og.Dense(A)
    eps = 1e-6
    res = ob.baca(g, n, eps, seed=0)
    t = res["trace"][0]
    _, R, P = scipy.linalg.qr(A, pivoting=True, mode="economic")
    rr = int(np.sum(np.abs(np.diag(R)) >= eps * abs(R[0, 0])))
    assert t["dk"] == rr
    kept = [t["J"][p] for p in t["jbar"]]
    assert kept == list(P[:rr])


@pytest.mark.parametrize("cplx", [False, True])
def test_product_of_random_exact_rank(cplx):
    """Product-of-random kernel (Sec. 5, kernel 6): rank exactly r after
    re-compression, error at rounding level."""
    U0, V0 = inputs.lowrank(11, 150, 130, 13, complex_=cplx)
    g = og.LowRank(U0, V0)
    res = ob.baca(g, 8, 1e-10, seed=1)
    U, s, V = ob.recompress(res["U"], res["V"], 1e-10)
    assert len(s) == 13
    A = U0 @ V0
    assert np.linalg.norm(A - (U * s) @ V) <= 1e-13 * np.linalg.norm(A)


def test_baca_cross_property():
    """(LRID2): after each iteration the residual vanishes on the kept
    columns, and on the kept rows when d_k = d."""
    g = _gauss_small()
    A = g(np.arange(g.m), np.arange(g.n))
    res = ob.baca(g, 6, 1e-12, seed=2)
    U, V = res["U"], res["V"]
    r = 0
    for t in res["trace"]:
        r += t["dk"]
        E = A - U[:, :r] @ V[:r]
        cols = [t["J"][p] for p in t["jbar"]]
        assert np.abs(E[:, cols]).max() < 1e-11
        if t["dk"] == len(t["I"]):
            assert np.abs(E[t["I"], :]).max() < 1e-11


def test_recompress_is_truncated_svd_of_product():
    rng = np.random.default_rng(12)
    U = rng.standard_normal((60, 9)) * np.geomspace(1, 1e-8, 9)
    V = rng.standard_normal((9, 50))
    Ur, s, Vr = ob.recompress(U, V, 1e-5)
    sv = np.linalg.svd(U @ V, compute_uv=False)
    assert len(s) == ol.eps_rank(sv, 1e-5)
    np.testing.assert_allclose(s, sv[:len(s)], rtol=1e-9)
    np.testing.assert_allclose(Ur.conj().T @ Ur, np.eye(len(s)), atol=1e-12)
    np.testing.assert_allclose(Vr @ Vr.conj().T, np.eye(len(s)), atol=1e-12)


# ---------------------------------------------------------------- merges / H-BACA
def _random_svd(rng, m, n, r, cplx):
    L = rng.standard_normal((m, r))
    R = rng.standard_normal((r, n))
    if cplx:
        L = L + 1j * rng.standard_normal((m, r))
        R = R + 1j * rng.standard_normal((r, n))
    A = L @ R
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    return U[:, :r], s[:r], Vh[:r], A


@pytest.mark.parametrize("cplx", [False, True])
def test_merges_equal_svd_of_concatenation(cplx):
    rng = np.random.default_rng(13)
    U1, s1, V1, A1 = _random_svd(rng, 30, 20, 4, cplx)
    U2, s2, V2, A2 = _random_svd(rng, 30, 25, 5, cplx)
    U, s, V = oh.horizontal_merge(U1, s1, V1, U2, s2, V2, 1e-12)
    sv = np.linalg.svd(np.concatenate([A1, A2], 1), compute_uv=False)
    np.testing.assert_allclose(s, sv[:len(s)], rtol=1e-10)
    np.testing.assert_allclose((U * s) @ V, np.concatenate([A1, A2], 1), atol=1e-10)
    U3, s3, V3, A3 = _random_svd(rng, 22, 20, 3, cplx)
    U, s, V = oh.vertical_merge(U1, s1, V1, U3, s3, V3, 1e-12)
    sv = np.linalg.svd(np.concatenate([A1, A3], 0), compute_uv=False)
    np.testing.assert_allclose(s, sv[:len(s)], rtol=1e-10)
    np.testing.assert_allclose((U * s) @ V, np.concatenate([A1, A3], 0), atol=1e-10)


def test_tree_split_sizes():
    lv = oh.tree_levels(2000, 2)
    assert lv[0] == [(0, 500), (500, 500), (1000, 500), (1500, 500)]
    lv = oh.tree_levels(50000, 5)
    sizes = [s for _, s in lv[0]]
    assert len(sizes) == 32 and sum(sizes) == 50000 and set(sizes) <= {1562, 1563}
    lv = oh.tree_levels(7, 2)
    assert [s for _, s in lv[0]] == [2, 2, 2, 1]


def test_hbaca_nb1_is_baca_plus_recompression():
    """Sec. 4: with n_b = 1 H-BACA is BACA (plus its re-compression)."""
    g = _gauss_small()
    h = oh.hbaca(g, 0, 8, 1e-8, seed=4)
    b = ob.baca(g, 8, 1e-8, seed=4, bid=osamp.block_id(0, 0, 0))
    U, s, V = ob.recompress(b["U"], b["V"], 1e-8)
    np.testing.assert_allclose(h["s"], s, rtol=1e-12)
    np.testing.assert_allclose((h["U"] * h["s"]) @ h["V"], (U * s) @ V, atol=1e-13)


@pytest.mark.parametrize("L", [0, 1, 2])
@pytest.mark.parametrize("eps", [1e-2, 1e-6, 1e-10])
def test_hbaca_accuracy_against_dense_svd(L, eps):
    """Sec. 5.2: error ~ eps with a slight increase as n_b grows; the rank is
    at least what Eckart-Young requires for the achieved 2-norm error."""
    x, y = inputs.gaussian_pair(seed=0, m=256, n=240)
    g = og.Gaussian(x, y, 1.0)
    res = oh.hbaca(g, L, 8, eps, seed=0)
    A = g(np.arange(g.m), np.arange(g.n))
    E = A - (res["U"] * res["s"]) @ res["V"]
    err = np.linalg.norm(E) / np.linalg.norm(A)
    sv = np.linalg.svd(A, compute_uv=False)
    # the eps-rank rule of Sec. 2 is relative to sigma_1, so even the exact
    # truncated SVD has Frobenius error e_opt = ||sigma_{r_eps+1:}|| / ||A||_F
    e_opt = np.linalg.norm(sv[ol.eps_rank(sv, eps):]) / np.linalg.norm(sv)
    assert err <= (1.1 if L == 0 else 2.0) * max(eps, e_opt)
    e2 = np.linalg.norm(E, 2)
    need = int(np.sum(sv > e2 * (1 + 1e-9)))
    assert res["r"] >= need
    if e2 < eps * sv[0]:
        assert res["r"] >= ol.eps_rank(sv, eps)


def test_hbaca_complex_helmholtz_small():
    x, y = inputs.sphere_pair(seed=1, m=300, n=280)
    g = og.Helmholtz(x, y, 4 * np.pi)
    res = oh.hbaca(g, 1, 16, 1e-4, seed=1)
    err = oapply.rel_error_dense(g, res["U"], res["s"], res["V"])
    assert err <= 2e-4
    A = g(np.arange(g.m), np.arange(g.n))
    sv = np.linalg.svd(A, compute_uv=False)
    assert res["r"] >= int(np.sum(sv > np.linalg.norm(A - (res["U"] * res["s"]) @ res["V"], 2)))


def test_rel_error_dense_against_direct_norm():
    """The chunked error evaluator equals ||A - U S V||_F / ||A||_F formed
    directly (row chunks smaller than m, so the chunk loop runs several
    times), on all rows and on a sample of rows."""
    rng = np.random.default_rng(4)
    x, y = inputs.gaussian_pair(seed=3, m=257, n=131)
    g = og.Gaussian(x, y, 0.9)
    A = g(np.arange(g.m), np.arange(g.n))
    Uf, sf, Vf = np.linalg.svd(A, full_matrices=False)
    U, s, V = Uf[:, :6], sf[:6] * (1 + 1e-3 * rng.standard_normal(6)), Vf[:6]
    want = np.linalg.norm(A - (U * s) @ V) / np.linalg.norm(A)
    assert abs(oapply.rel_error_dense(g, U, s, V, row_chunk=50) - want) <= 1e-13 * want
    I = np.sort(rng.choice(g.m, 40, replace=False))
    want_I = np.linalg.norm(A[I] - (U[I] * s) @ V) / np.linalg.norm(A[I])
    assert abs(oapply.rel_error_dense(g, U, s, V, row_chunk=16, rows=I) - want_I) <= 1e-13 * want_I
    # a closed form: U S V = truncated SVD gives the tail of the singular values
    tail = np.sqrt(np.sum(sf[6:] ** 2) / np.sum(sf ** 2))
    assert abs(oapply.rel_error_dense(g, Uf[:, :6], sf[:6], Vf[:6], row_chunk=64) - tail) <= 1e-12


class _UlpPerturbed:
    """A generator whose entries differ from ``gen``'s by -1, 0 or +1 unit in
    the last place (a fixed pattern): an input change at the rounding level."""

    def __init__(self, gen):
        self.gen, self.m, self.n, self.dtype = gen, gen.m, gen.n, gen.dtype

    def __call__(self, I, J):
        A = self.gen(I, J)
        I, J = np.asarray(I), np.asarray(J)
        return A + ((I[:, None] * 7919 + J[None, :] * 104729) % 3 - 1) * np.spacing(A)


def test_coherent_case_is_rounding_sensitive():
    """On the coherent sparse product (the benchmark's 6000^2 shape, d = 32,
    eps = 1e-8) BACA reaches crosses at the rounding level and the LRID
    triangle amplifies rounding by up to 1/eps: a 1-ulp change of the input
    changes a leaf's BACA rank by more than 2 and its error by far more than
    1e-10, in the oracle itself.  So two correct implementations cannot be
    held to rank +-2 and error 1e-10 on this input past such a cross (the GPU
    tests compare the prefix before it).  The smooth Gaussian kernel under the
    same perturbation keeps its rank and its error to 1e-12."""
    sp = inputs.sparse_product(seed=2, m=6000, n=6000, K=50, density=0.01)
    g = og.SparseProduct(sp.dense_P(), sp.dense_Q(), sp.P2, sp.Q2)
    gp = _UlpPerturbed(g)
    rows = oh.tree_levels(6000, 2)[0]
    worst_rank, worst_err = 0, 0.0
    for b in range(4):
        res = []
        for gen in (g, gp):
            w = og.Window(gen, rows[0][0], rows[0][1], rows[b][0], rows[b][1])
            r = ob.baca(w, 32, 1e-8, seed=2, bid=osamp.block_id(0, 0, b))
            A = og.Window(g, rows[0][0], rows[0][1], rows[b][0], rows[b][1])(np.arange(1500), np.arange(1500))
            res.append((r["r"], np.linalg.norm(A - r["U"] @ r["V"]) / np.linalg.norm(A)))
        worst_rank = max(worst_rank, abs(res[0][0] - res[1][0]))
        worst_err = max(worst_err, abs(res[0][1] - res[1][1]))
    assert worst_rank > 2 and worst_err > 1e-6, (worst_rank, worst_err)
    x, y = inputs.gaussian_pair(seed=0, m=600, n=520)
    gg = og.Gaussian(x, y, 1.0)
    r0, r1 = oh.hbaca(gg, 1, 8, 1e-8, seed=0), oh.hbaca(_UlpPerturbed(gg), 1, 8, 1e-8, seed=0)
    A = gg(np.arange(600), np.arange(520))
    e0 = np.linalg.norm(A - (r0["U"] * r0["s"]) @ r0["V"]) / np.linalg.norm(A)
    e1 = np.linalg.norm(A - (r1["U"] * r1["s"]) @ r1["V"]) / np.linalg.norm(A)
    assert r0["r"] == r1["r"] and abs(e0 - e1) <= 1e-12 * max(e0, 1e-300) + 1e-15


@pytest.mark.parametrize("cplx", [False, True])
def test_baca_with_strong_rrqr_pivots(cplx):
    """BACA with strong-RRQR pivot sets (f = 1.05): exact rank and rounding
    error on a product of random factors, the cross property on the kept
    columns, and the frozen replay of its own record valid (sets without a
    swap above f^2 left)."""
    LU, LV = inputs.lowrank(21, 160, 150, 11, complex_=cplx)
    g = og.LowRank(LU, LV)
    res = ob.baca(g, 8, 1e-10, seed=3, srrqr_f=1.05)
    A = LU @ LV
    assert len(ob.recompress(res["U"], res["V"], 1e-10)[1]) == 11
    assert np.linalg.norm(A - res["U"] @ res["V"]) <= 1e-12 * np.linalg.norm(A)
    rep = ob.baca_replay(g, 8, 1e-10, res["trace"], seed=3, stop=res["stop"], srrqr_f=1.05)
    for r in rep["recs"]:
        if r.get("noise_level"):
            break
        assert r["valid_I"] and r["valid_J"] and r["valid_W"] and r["valid_dk"], r
    x, y = inputs.gaussian_pair(seed=9, m=300, n=280)
    gg = og.Gaussian(x, y, 0.6)
    res = ob.baca(gg, 8, 1e-9, seed=1, srrqr_f=1.0)
    E = gg(np.arange(300), np.arange(280)) - res["U"] @ res["V"]
    kept = [t["J"][p] for t in res["trace"] for p in t["jbar"]]
    assert np.abs(E[:, kept]).max() <= 1e-10 * np.abs(E).max() + 1e-14
    assert sum(sum(t["swaps"]) for t in res["trace"]) > 0  # the refinement acted


# ---------------------------------------------------------------- frozen-pivot replay
@pytest.mark.parametrize("cplx", [False, True])
def test_replay_of_own_trace_is_valid_and_identical(cplx):
    if cplx:
        x, y = inputs.sphere_pair(seed=4, m=160, n=150)
        g = og.Helmholtz(x, y, 4 * np.pi)
    else:
        g = _gauss_small()
    res = ob.baca(g, 6, 1e-9, seed=5)
    rep = ob.baca_replay(g, 6, 1e-9, res["trace"], seed=5)
    for r in rep["recs"]:
        assert r["J_ok"] and r["valid_I"] and r["valid_J"] and r["valid_W"] and r["valid_dk"] and r["valid_stop"], r
    assert rep["r"] == res["r"]
    np.testing.assert_allclose(rep["U"] @ rep["V"], res["U"] @ res["V"], rtol=0, atol=1e-13)
    for a, b in zip(rep["recs"], res["trace"]):
        assert abs(a["nu"] - b["nu"]) <= 1e-12 * b["mu"] and abs(a["mu"] - b["mu"]) <= 1e-12 * b["mu"]


def test_replay_flags_a_non_greedy_pivot():
    g = _gauss_small()
    res = ob.baca(g, 6, 1e-9, seed=5)
    bad = [dict(t) for t in res["trace"]]
    # swap the first two row pivots of the first iteration: the second is not the max at step 0
    bad[0] = dict(bad[0], I=[bad[0]["I"][1], bad[0]["I"][0]] + bad[0]["I"][2:])
    rep = ob.baca_replay(g, 6, 1e-9, bad, seed=5)
    assert not rep["recs"][0]["valid_I"]
    # a kept row reused later is not a candidate
    bad = [dict(t) for t in res["trace"]]
    bad[1] = dict(bad[1], I=[res["trace"][0]["I"][0]] + bad[1]["I"][1:])
    rep = ob.baca_replay(g, 6, 1e-9, bad, seed=5)
    assert not rep["recs"][1]["valid_I"]
    # a wrong rank decision d_k is flagged
    bad = [dict(t) for t in res["trace"]]
    bad[0] = dict(bad[0], dk=bad[0]["dk"] - 1, jbar=bad[0]["jbar"][:-1])
    rep = ob.baca_replay(g, 6, 1e-9, bad, seed=5)
    assert not rep["recs"][0]["valid_dk"]


def test_replay_with_full_blocks_is_the_skeleton_approximation():
    """With every kept block full (d_k = d), the cross approximation after K
    iterations is the skeleton A(:, J*) A(I*, J*)^-1 A(I*, :) over the kept
    rows I* and columns J* (Alg. 2 is a block partial LU): the identity the
    frozen-pivot reverse pass rests on."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (80, 3))
    y = rng.uniform(0, 1, (70, 3)) + np.array([1.5, 0.0, 0.0])
    g = og.Gaussian(x, y, 0.6)
    d = 4
    r = ob.baca(g, d, 1e-13, seed=0, bid=0)
    K = 0
    for t in r["trace"]:
        if t["dk"] != d or len(t["I"]) != d:
            break
        K += 1
    K = min(K, 3)
    assert K >= 2
    rep = ob.baca_replay(g, d, 1e-13, r["trace"][:K], seed=0, bid=0, stop="iterations")
    Istar = [i for t in r["trace"][:K] for i in t["I"][:t["dk"]]]
    Jstar = [t["J"][p] for t in r["trace"][:K] for p in t["jbar"][:t["dk"]]]
    A = g(np.arange(g.m), np.arange(g.n))
    skel = A[:, Jstar] @ np.linalg.solve(A[np.ix_(Istar, Jstar)], A[Istar, :])
    assert np.linalg.norm(rep["U"] @ rep["V"] - skel) <= 1e-9 * np.linalg.norm(A)
    # and it is not the trivial case: A itself is not reproduced yet
    assert np.linalg.norm(A - skel) > 1e-6 * np.linalg.norm(A)


def test_frozen_truncation_rank_reproduces_eps_rank():
    """H-BACA with every truncation rank frozen at the ranks an unfrozen run
    took is the same computation; a smaller frozen rank truncates further."""
    x, y = inputs.gaussian_pair(seed=4, m=240, n=200)
    g = og.Gaussian(x, y, 0.7)
    a = oh.hbaca(g, 1, 8, 1e-8, seed=0)
    b = oh.hbaca(g, 1, 8, 1e-8, seed=0, ranks=a["ranks"])
    assert a["r"] == b["r"]
    np.testing.assert_array_equal(a["s"], b["s"])
    root = ("full", 1, 0, 0)
    c = oh.hbaca(g, 1, 8, 1e-8, seed=0, ranks={root: a["r"] - 3})
    assert c["r"] == a["r"] - 3
    np.testing.assert_allclose(c["s"], a["s"][:a["r"] - 3], rtol=1e-12)
