"""GPU parity of the batched form: many independent Gaussian-kernel blocks of
uneven sizes, each with its own tree depth, compressed by one
hbaca_compress_batched call and checked block by block against the oracle
H-BACA (Alg. 3) run with the same J_1 streams (batch index = block number).
Needs a GB300."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import baca as ob
from oracle import generators as og
from oracle import hbaca as oh
from oracle import linalg as ol
from oracle import sampler as osamp
from paper_1901_06101_gb300 import binding as B
from paper_1901_06101_gb300 import inputs
from tests.parity import check_leaf_replay, near_threshold
from tests.test_gpu_parity import check_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return B.Context()


def levels_for(m, n, target):
    """Tree depth for a leaf target of `target` rows/columns: the smallest L
    with ceil(max(m, n) / 2^L) <= target, lowered until 2^L <= min(m, n)."""
    L = 0
    while -(-max(m, n) // (1 << L)) > target:
        L += 1
    while L > 0 and (1 << L) > min(m, n):
        L -= 1
    return L


def _specs(blocks):
    return [B.gaussian(x, y, h) for (x, y, h) in blocks]


def test_batched_matches_oracle_per_block(ctx):
    blocks = inputs.batched_blocks(seed=3, nblocks=12, lo=64, hi=700)
    d, eps, target, seed = 8, 1e-8, 256, 0
    specs = _specs(blocks)
    opts = B.make_opts(eps, d, -target, seed=seed, rank_cap=256, leaf_rank_cap=256)
    outs = B.compress_batched(ctx, specs, opts)
    torch.cuda.synchronize()
    depths = set()
    for b, ((x, y, h), res) in enumerate(zip(blocks, outs)):
        ogen = og.Gaussian(x, y, h)
        L = levels_for(ogen.m, ogen.n, target)
        depths.add(L)
        rows = oh.tree_levels(ogen.m, L)[0]
        cols = oh.tree_levels(ogen.n, L)[0]
        nb = 1 << L
        traces = {}
        for leaf in range(nb * nb):
            a, c = divmod(leaf, nb)
            w = og.Window(ogen, rows[a][0], rows[a][1], cols[c][0], cols[c][1])
            g = B.read_leaf_trace_batched(specs, opts, outs[0].ws, b, leaf)
            traces[leaf] = g
            rep = check_leaf_replay(w, g, d, eps, seed, osamp.block_id(b, a, c))
            if not rep["comparable"]:
                continue
            Uo, so, Vo = ob.recompress(rep["U"], rep["V"], eps)
            sv_all = np.linalg.svd(rep["U"] @ rep["V"], compute_uv=False) if rep["r"] else np.zeros(0)
            if not near_threshold(sv_all, eps):
                assert g["rank"] == len(so), ("leaf rank", b, leaf, g["rank"], len(so))
        full = oh.hbaca(ogen, L, d, eps, seed=seed, batch_index=b, forced=traces)
        check_result(ogen, res, eps, full)
    assert len(depths) >= 2, depths


def test_batched_frob_budget_per_block(ctx):
    """HBACA_FLAG_FROB in a batch: every block's truncations take the budget
    of its own depth, eps / sqrt(2L + 1); each block against the oracle
    H-BACA with trunc="frob" at that depth."""
    blocks = inputs.batched_blocks(seed=3, nblocks=6, lo=64, hi=700)
    d, eps, target, seed = 8, 1e-8, 256, 0
    specs = _specs(blocks)
    opts = B.make_opts(eps, d, -target, seed=seed, rank_cap=256, leaf_rank_cap=256, flags=B.FLAG_FROB)
    outs = B.compress_batched(ctx, specs, opts)
    torch.cuda.synchronize()
    depths = set()
    for b, ((x, y, h), res) in enumerate(zip(blocks, outs)):
        ogen = og.Gaussian(x, y, h)
        L = levels_for(ogen.m, ogen.n, target)
        depths.add(L)
        nb = 1 << L
        traces = {leaf: B.read_leaf_trace_batched(specs, opts, outs[0].ws, b, leaf) for leaf in range(nb * nb)}
        full = oh.hbaca(ogen, L, d, eps, seed=seed, batch_index=b, forced=traces, trunc="frob")
        check_result(ogen, res, eps, full)
    assert len(depths) >= 2, depths


def test_batched_single_block_equals_compress(ctx):
    """A batch of one is the plain call: same plan, same streams, same bits."""
    x, y = inputs.gaussian_pair(seed=4, m=777, n=650)
    spec = B.gaussian(x, y, 0.8)
    opts = B.make_opts(1e-8, 8, 1, seed=2, rank_cap=200, leaf_rank_cap=256)
    r1 = B.compress(ctx, spec, opts)
    r2 = B.compress_batched(ctx, [spec], opts)[0]
    torch.cuda.synchronize()
    assert r1.rank == r2.rank
    assert torch.equal(r1.S, r2.S)
    assert torch.equal(r1.U, r2.U)
    assert torch.equal(r1.V, r2.V)


def test_batched_error_bound_every_block(ctx):
    """Every block of a batch is within a factor 2 of the error of its own
    truncated SVD at the eps-rank (Eckart-Young; the eps-rank rule sigma >=
    eps sigma_1 alone can leave a Frobenius error above eps), or of eps."""
    blocks = inputs.batched_blocks(seed=7, nblocks=10, lo=64, hi=500)
    opts = B.make_opts(1e-8, 8, -256, seed=1, rank_cap=256, leaf_rank_cap=256)
    outs = B.compress_batched(ctx, _specs(blocks), opts)
    torch.cuda.synchronize()
    for b, ((x, y, h), res) in enumerate(zip(blocks, outs)):
        ogen = og.Gaussian(x, y, h)
        A = ogen(np.arange(ogen.m), np.arange(ogen.n))
        U, S, V = res.U.cpu().numpy(), res.S.cpu().numpy(), res.V.cpu().numpy()
        err = np.linalg.norm(A - (U * S) @ V) / np.linalg.norm(A)
        sv = np.linalg.svd(A, compute_uv=False)
        e_opt = np.linalg.norm(sv[ol.eps_rank(sv, 1e-8):]) / np.linalg.norm(sv)
        assert err <= 2 * max(1e-8, e_opt), (b, err, e_opt)


def test_batched_rejects_mixed_kinds(ctx):
    x, y = inputs.gaussian_pair(seed=0, m=100, n=100)
    specs = [B.gaussian(x, y, 1.0), B.helmholtz(x, y, 1.0)]
    opts = B.make_opts(1e-8, 8, 0)
    with pytest.raises(B.HbacaError):
        B.compress_batched(ctx, specs, opts)


def _same_results(a, b):
    for ra, rb in zip(a.results(), b.results()):
        assert ra.rank == rb.rank
        assert torch.equal(ra.S, rb.S) and torch.equal(ra.U, rb.U) and torch.equal(ra.V, rb.V)


def test_explicit_leaf_cluster_and_workspace_checks(ctx):
    """A batch with a fixed leaf cluster size gets a workspace planned for
    that size and the same factors as the automatic choice (the cluster size
    never changes a result); a workspace or output buffer smaller than the
    plan needs is refused before anything is launched."""
    blocks = inputs.batched_blocks(seed=13, nblocks=12, lo=64, hi=600)
    specs = _specs(blocks)
    mk = lambda c: B.make_opts(1e-8, 8, -256, seed=0, rank_cap=256, leaf_rank_cap=256, cluster=c)
    auto = B.Batch(ctx, specs, mk(0)).run()
    for c in (1, 16):
        one = B.Batch(ctx, specs, mk(c)).run()
        torch.cuda.synchronize()
        _same_results(auto, one)
    small = torch.empty(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.HbacaError):
        B.Batch(ctx, specs, mk(1), ws=small).run()
    with pytest.raises(B.HbacaError):
        B.compress(ctx, specs[0], mk(0), ws=small)
    s0 = specs[0]
    tiny = (torch.empty((1, s0.m), dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty((1, s0.n), dtype=torch.float64, device="cuda"))
    with pytest.raises(B.HbacaError):
        B.compress(ctx, s0, mk(0), out=tiny)


def test_graph_replay_bit_identical_and_follows_new_data(ctx):
    """HBACA_FLAG_GRAPH: the first call runs and captures itself, later calls
    replay the graph; every replay equals a plain call bit for bit, also after
    the points change in place (same buffers, new data)."""
    blocks = inputs.batched_blocks(seed=11, nblocks=24, lo=64, hi=600)
    specs = _specs(blocks)
    plain = B.make_opts(1e-8, 8, -256, seed=0, rank_cap=256, leaf_rank_cap=256)
    gopts = B.make_opts(1e-8, 8, -256, seed=0, rank_cap=256, leaf_rank_cap=256, flags=B.FLAG_GRAPH)
    gctx = B.Context()
    ref = B.Batch(ctx, specs, plain).run()
    gb = B.Batch(gctx, specs, gopts)
    for _ in range(3):
        gb.run()
        torch.cuda.synchronize()
        _same_results(ref, gb)
    for s in specs:  # new points in the same device buffers
        s.keep[0].mul_(1.05)
        s.keep[1].add_(0.02)
    ref2 = B.Batch(ctx, specs, plain).run()
    gb.run()
    torch.cuda.synchronize()
    _same_results(ref2, gb)


def test_autotune_returns_a_cluster_size_with_valid_results(ctx):
    blocks = inputs.batched_blocks(seed=12, nblocks=16, lo=64, hi=600)
    specs = _specs(blocks)
    opts = B.make_opts(1e-8, 8, -256, seed=0, rank_cap=256, leaf_rank_cap=256)
    bt = B.Batch(ctx, specs, opts)
    c, ms = bt.autotune()
    assert c in (1, 2, 4, 8, 16) and ms > 0
    bt.run()
    torch.cuda.synchronize()
    for (x, y, h), res in zip(blocks, bt.results()):
        ogen = og.Gaussian(x, y, h)
        A = ogen(np.arange(ogen.m), np.arange(ogen.n))
        U, S, V = res.U.cpu().numpy(), res.S.cpu().numpy(), res.V.cpu().numpy()
        err = np.linalg.norm(A - (U * S) @ V) / np.linalg.norm(A)
        sv = np.linalg.svd(A, compute_uv=False)
        e_opt = np.linalg.norm(sv[ol.eps_rank(sv, 1e-8):]) / np.linalg.norm(sv)
        assert err <= 2 * max(1e-8, e_opt), (err, e_opt)


def test_graph_replay_of_a_single_block_with_cluster_groups(ctx):
    """HBACA_FLAG_GRAPH on one 2000^2 block at L = 2: the root stage spreads
    its QR and Q application over several clusters (a cooperative launch and
    counter resets inside the graph) and stages with several Jacobi groups fork
    a second stream; every replay equals the plain call bit for bit."""
    x, y = inputs.gaussian_pair(seed=0, m=2000, n=2000)
    spec = B.gaussian(x, y, 1.0)
    plain = B.make_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256)
    ref = B.compress(ctx, spec, plain)
    torch.cuda.synchronize()
    gopts = B.make_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256, flags=B.FLAG_GRAPH)
    gctx = B.Context()
    ws = torch.empty(B.workspace_size(spec.gen, gopts), dtype=torch.uint8, device="cuda")
    first = B.compress(gctx, spec, gopts, ws=ws)
    torch.cuda.synchronize()
    for r in [first] + [B.compress(gctx, spec, gopts, ws=ws, out=first.buffers) for _ in range(3)]:
        torch.cuda.synchronize()
        assert r.rank == ref.rank
        assert torch.equal(r.S, ref.S) and torch.equal(r.U, ref.U) and torch.equal(r.V, ref.V)
