"""The paper's Polynomial (Sec. 5, kernel 5) and EFIE2D (Sec. 5, kernel 2)
generators on the GPU: their entries against the oracle's, then H-BACA
parity through the C ABI (pivots while unique, frozen-pivot replay, final
factors against the frozen-pivot oracle).  Needs a GB300."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import generators as og
from oracle import hbaca as oh
from paper_1901_06101_gb300 import binding as B
from paper_1901_06101_gb300 import inputs
from tests.test_gpu_parity import check_result, compare_with_frozen_oracle, run_and_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return B.Context()


def test_hankel_entries_against_scipy(ctx):
    """H0^(2)(k r) over arguments from 1e-6 to 5000 (both branches of the
    device function: series from Miller's recurrence below 20, Hankel's
    expansion above), relative to the amplitude max(|H0|, sqrt(2/(pi z)))."""
    z = np.concatenate([np.geomspace(1e-6, 1.0, 300), np.linspace(1.0, 40.0, 3000), np.geomspace(40.0, 5000.0, 700)])
    x = np.zeros((1, 2))
    y = np.stack([z, np.zeros_like(z)], axis=1)
    spec = B.hankel2d(x, y, 1.0)
    got = B.entries(spec, np.zeros(z.size, np.int64), np.arange(z.size))
    want = og.Hankel2D(x, y, 1.0)([0], np.arange(z.size))[0]
    env = np.maximum(np.abs(want), np.sqrt(2.0 / (np.pi * z)))
    err = np.abs(got - want) / env
    assert err.max() <= 1e-13, (err.max(), z[np.argmax(err)])


def test_polynomial_and_strip_entries(ctx):
    rng = np.random.default_rng(0)
    x, y = inputs.polynomial_pair(seed=3, m=300, n=250, dim=50)
    I, J = rng.integers(0, 300, 500), rng.integers(0, 250, 500)
    got = B.entries(B.polynomial(x, y, 0.7), I, J)
    want = og.Polynomial(x, y, 0.7)(I, J)[np.arange(500), np.arange(500)]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    xs, ys, k = inputs.strips_pair(600)
    I, J = rng.integers(0, 600, 500), rng.integers(0, 600, 500)
    got = B.entries(B.hankel2d(xs, ys, k), I, J)
    want = og.Hankel2D(xs, ys, k)(I, J)[np.arange(500), np.arange(500)]
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-12


def test_polynomial_exact_rank(ctx):
    """dim = 5: the kernel has rank 1 + 5 + 15 = 21 exactly; H-BACA must find
    it, with error at the rounding level."""
    x, y = inputs.polynomial_pair(seed=5, m=1400, n=1300, dim=5)
    spec = B.polynomial(x, y, 0.4)
    ogen = og.Polynomial(x, y, 0.4)
    res, compared, div, tr = run_and_compare(ctx, spec, ogen, 2, 8, 1e-12, seed=2)
    assert res.rank == 21
    full = oh.hbaca(ogen, 2, 8, 1e-12, seed=2, forced=tr)
    check_result(ogen, res, 1e-12, full)


def test_polynomial_dim50(ctx):
    """The paper's polynomial kernel with points in R^50 (h = 1, eps = 1e-3,
    d = 16, 2 x 2 leaves of 1000^2: eps-rank about 320 of at most 1326)."""
    x, y = inputs.polynomial_pair(seed=6, m=2000, n=2000, dim=50)
    spec = B.polynomial(x, y, 1.0)
    ogen = og.Polynomial(x, y, 1.0)
    res, compared, div, tr = run_and_compare(ctx, spec, ogen, 1, 16, 1e-3, seed=4, rank_cap=1024, leaf_cap=1000)
    full = oh.hbaca(ogen, 1, 16, 1e-3, seed=4, forced=tr)
    compare_with_frozen_oracle(res, full, ogen, tr)


def test_polynomial_dim20_exact_rank(ctx):
    """dim = 20: rank 1 + 20 + 210 = 231 exactly, recovered at eps = 1e-10."""
    x, y = inputs.polynomial_pair(seed=8, m=1600, n=1500, dim=20)
    spec = B.polynomial(x, y, 1.0)
    ogen = og.Polynomial(x, y, 1.0)
    res, compared, div, tr = run_and_compare(ctx, spec, ogen, 1, 16, 1e-10, seed=5, rank_cap=512, leaf_cap=512)
    assert res.rank == 231
    full = oh.hbaca(ogen, 1, 16, 1e-10, seed=5, forced=tr)
    check_result(ogen, res, 1e-10, full)


def test_efie2d_strips(ctx):
    """EFIE2D between two parallel strips of length 1 at distance 1, 15 points
    per wavelength (2000 points each, k = 838), eps = 1e-6, d = 16, 4 x 4
    leaves."""
    x, y, k = inputs.strips_pair(2000)
    spec = B.hankel2d(x, y, k)
    ogen = og.Hankel2D(x, y, k)
    # the points form regular grids: column norms tie exactly, so the free
    # pivot comparison ends early; the frozen-pivot replay covers every leaf
    res, compared, div, tr = run_and_compare(ctx, spec, ogen, 2, 16, 1e-6, seed=7, rank_cap=512, leaf_cap=512)
    full = oh.hbaca(ogen, 2, 16, 1e-6, seed=7, forced=tr)
    check_result(ogen, res, 1e-6, full)
    assert abs(B.rel_error(ctx, spec, res) - oapply_err(ogen, res)) <= 1e-12


def oapply_err(ogen, res):
    from oracle import apply as oapply
    return oapply.rel_error_dense(ogen, res.U.cpu().numpy(), res.S.cpu().numpy(), res.V.cpu().numpy(), row_chunk=256)
