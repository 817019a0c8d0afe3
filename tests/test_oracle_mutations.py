"""Plant plausible mistakes in the oracle (CPU only) and check that the pins
in test_oracle_pins catch each one."""
import numpy as np
import pytest
import scipy.linalg

from oracle import apply as oapply
from oracle import baca as ob
from oracle import hbaca as oh
from oracle import linalg as ol
from tests import test_oracle_pins as pins


def _expect_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_dropped_cross_term_in_lrnormup(monkeypatch):
    def bad(U, V, mu, Uk, Vk, nu):
        return float(np.sqrt(mu * mu + nu * nu))
    monkeypatch.setattr(ob, "lrnormup", bad)
    _expect_failure(pins.test_lrnorm_and_update_identities, False)


def test_transpose_instead_of_adjoint_in_lrid(monkeypatch):
    def bad(C, W, R, eps):
        dI, dJ = W.shape
        piv, diag, _, Q = ol.greedy_qrcp(W, min(dI, dJ), rank_tol=eps)
        T = np.triu(Q.T @ W[:, piv])
        return C[:, piv], scipy.linalg.solve_triangular(T, Q.T @ R), len(piv), piv
    monkeypatch.setattr(ob, "lrid", bad)
    _expect_failure(pins.test_lrid_is_interpolative_decomposition, True)


def test_missing_sigma_in_horizontal_merge(monkeypatch):
    orig = oh.horizontal_merge
    def bad(U1, s1, V1, U2, s2, V2, eps):
        return orig(U1, np.ones_like(s1), V1, U2, np.ones_like(s2), V2, eps)
    monkeypatch.setattr(oh, "horizontal_merge", bad)
    _expect_failure(pins.test_merges_equal_svd_of_concatenation, False)


def test_wrong_rank_rule(monkeypatch):
    monkeypatch.setattr(ol, "eps_rank", lambda s, eps: int(np.count_nonzero(np.asarray(s) > eps)))
    _expect_failure(pins.test_eps_rank_definition)


def test_qrcp_without_projection(monkeypatch):
    def bad(Q, X):
        return X.copy()
    monkeypatch.setattr(ol, "_project_out", bad)
    _expect_failure(pins.test_greedy_qrcp_matches_lapack_geqp3, False)


def test_recompress_with_dropped_conjugate(monkeypatch):
    def bad(U, V, eps):
        Qu, Tu = np.linalg.qr(U)
        Qv, Tv = np.linalg.qr(V.conj().T)
        X, s, Yh = ol.truncated_svd(Tu @ Tv.conj().T, eps)
        return Qu @ X, s, Yh @ Qv.T
    monkeypatch.setattr(ob, "recompress", bad)
    _expect_failure(pins.test_product_of_random_exact_rank, True)


def test_qrcp_noise_residual_adds_no_direction(monkeypatch):
    """A basis that skips chosen columns whose residual is at the rounding
    level no longer spans the chosen columns."""
    orig = ol.greedy_qrcp

    def bad(M, kmax, **kw):
        out = orig(M, kmax, **kw)
        piv, diag, marg, Q = out[:4]
        Q = Q.copy()
        for t, dv in enumerate(diag):
            if dv < 1e-12 * diag[0]:
                Q[:, t] = 0.0
        return (piv, diag, marg, Q) + tuple(out[4:])
    monkeypatch.setattr(ol, "greedy_qrcp", bad)
    _expect_failure(pins.test_greedy_qrcp_basis_spans_the_chosen_columns)


def test_rel_error_without_square_root(monkeypatch):
    orig = oapply.rel_error_dense
    monkeypatch.setattr(oapply, "rel_error_dense", lambda *a, **k: orig(*a, **k) ** 2)
    _expect_failure(pins.test_rel_error_dense_against_direct_norm)


def test_rel_error_last_chunk_dropped(monkeypatch):
    def bad(gen, U, s, V, row_chunk=2048, rows=None):
        allrows = np.arange(gen.m) if rows is None else np.asarray(rows)
        keep = allrows[: max(row_chunk, (allrows.size // row_chunk) * row_chunk)]
        A = gen(keep, np.arange(gen.n))
        return float(np.linalg.norm(A - (U[keep] * s) @ V) / np.linalg.norm(A))
    monkeypatch.setattr(oapply, "rel_error_dense", bad)
    _expect_failure(pins.test_rel_error_dense_against_direct_norm)


def test_hankel_of_the_first_kind(monkeypatch):
    import scipy.special
    monkeypatch.setattr(scipy.special, "hankel2", scipy.special.hankel1)
    _expect_failure(pins.test_hankel2d_generator_published_values)


def test_polynomial_without_square(monkeypatch):
    from oracle import generators as og
    monkeypatch.setattr(og.Polynomial, "__call__",
                        lambda self, I, J: self.x[np.asarray(I)] @ self.y[np.asarray(J)].T + self.h)
    _expect_failure(pins.test_polynomial_generator_closed_form_and_rank)


def test_strong_rrqr_criterion_without_residual_term(monkeypatch):
    orig = ol.strong_rrqr_criterion

    def bad(M, piv, rest):
        A = M[:, piv]
        Q, R11 = np.linalg.qr(A)
        Ri = scipy.linalg.solve_triangular(R11, np.eye(len(piv)), lower=False)
        return np.abs(Ri @ (Q.conj().T @ M[:, rest])) ** 2
    monkeypatch.setattr(ol, "strong_rrqr_criterion", bad)
    _expect_failure(pins.test_strong_rrqr_criterion_is_the_volume_ratio_of_a_swap, 9, 5)


def test_frob_budget_not_split_over_the_truncations(monkeypatch):
    monkeypatch.setattr(oh, "frob_budget", lambda eps, L: eps)
    _expect_failure(pins.test_hbaca_frob_truncations_follow_the_budget)


def test_frob_budget_split_linearly(monkeypatch):
    monkeypatch.setattr(oh, "frob_budget", lambda eps, L: eps / (2.0 * L + 1.0))
    _expect_failure(pins.test_hbaca_frob_truncations_follow_the_budget)


def test_frob_rank_off_by_one(monkeypatch):
    orig = ol.frob_rank
    monkeypatch.setattr(ol, "frob_rank", lambda s, e: max(orig(s, e) - 1, 0))
    _expect_failure(pins.test_frob_truncation_is_eckart_young_minimal, 1e-3)
