"""hbaca_compress_noalloc (workspace built into the library) against
hbaca_compress (workspace from the caller), through the C ABI, on the same
inputs and two calls in a row.  Needs a GB300.  Kept in its own module, named
to be collected last, so that it runs both alone and after the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1901_06101_gb300 import binding as B
from paper_1901_06101_gb300 import inputs

pytestmark = pytest.mark.gpu

HBACA_WORKSPACE = 7


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return B.Context()


def _same(ref, got):
    """The two calls run the same kernels with the same launch shapes on the
    same inputs, and every reduction has a fixed order: the factors are
    bit-identical."""
    assert got.rank == ref.rank
    assert torch.equal(got.U, ref.U) and torch.equal(got.S, ref.S) and torch.equal(got.V, ref.V)


def test_noalloc_matches_compress_two_calls(ctx):
    x, y = inputs.gaussian_pair(seed=0, m=600, n=520)
    spec = B.gaussian(x, y, 1.0)
    opts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=128, leaf_rank_cap=256)
    ref = B.compress(ctx, spec, opts)
    torch.cuda.synchronize()
    assert ref.rank > 0
    for _ in range(2):
        got = B.compress_noalloc(ctx, spec, opts)
        torch.cuda.synchronize()
        _same(ref, got)


def test_noalloc_other_problem_then_back(ctx):
    """A complex problem with another plan in between: the built-in area is
    reused and the first problem still gives the same result."""
    xs, ys = inputs.sphere_pair(seed=1, m=700, n=600)
    hspec = B.helmholtz(xs, ys, 4 * np.pi)
    hopts = B.make_opts(1e-4, 8, 1, seed=0, rank_cap=96, leaf_rank_cap=128)
    href = B.compress(ctx, hspec, hopts)
    x, y = inputs.gaussian_pair(seed=0, m=600, n=520)
    gspec = B.gaussian(x, y, 1.0)
    gopts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=128, leaf_rank_cap=256)
    gref = B.compress(ctx, gspec, gopts)
    torch.cuda.synchronize()
    for _ in range(2):
        _same(href, B.compress_noalloc(ctx, hspec, hopts))
        _same(gref, B.compress_noalloc(ctx, gspec, gopts))
    torch.cuda.synchronize()


def test_noalloc_rejects_problem_above_limit(ctx):
    x, y = inputs.gaussian_pair(seed=0, m=2000, n=2000)
    spec = B.gaussian(x, y, 1.0)
    opts = B.make_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256)
    with pytest.raises(B.HbacaError) as ei:
        B.compress_noalloc(ctx, spec, opts)
    assert ei.value.code == HBACA_WORKSPACE
    assert "built-in area" in str(ei.value)
    # nothing was enqueued; a problem that fits still runs
    x, y = inputs.gaussian_pair(seed=0, m=600, n=520)
    small = B.gaussian(x, y, 1.0)
    sopts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=128, leaf_rank_cap=256)
    _same(B.compress(ctx, small, sopts), B.compress_noalloc(ctx, small, sopts))


def test_noalloc_refuses_graph_and_tape(ctx):
    """A captured graph would replay against descriptor tables that later
    calls overwrite in the shared area, and a tape there cannot reach the
    reverse pass: both flags are refused before anything is enqueued."""
    x, y = inputs.gaussian_pair(seed=0, m=600, n=520)
    spec = B.gaussian(x, y, 1.0)
    for flag in (B.FLAG_GRAPH, B.FLAG_TAPE):
        opts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=128, leaf_rank_cap=256, flags=flag)
        with pytest.raises(B.HbacaError) as ei:
            B.compress_noalloc(ctx, spec, opts)
        assert ei.value.code == 1
    opts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=128, leaf_rank_cap=256)
    _same(B.compress(ctx, spec, opts), B.compress_noalloc(ctx, spec, opts))
