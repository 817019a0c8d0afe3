"""Plant plausible mistakes in the oracle (CPU only) and check that the pins
in test_oracle_pins catch each one."""
import numpy as np
import pytest
import scipy.linalg

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
