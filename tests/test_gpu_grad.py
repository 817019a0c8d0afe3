"""GPU parity of y = U(S(V X)) and of its reverse pass with frozen pivots
(hbaca_apply, hbaca_apply_backward) through the C ABI.  The reference
gradient is the central finite difference of the oracle H-BACA with the
GPU's pivots (frozen-pivot replay of every leaf) and the oracle's own
truncation ranks frozen; a second reference is autograd through the dense
kernel matrix, which differs from the gradient of the compressed map by
O(eps).  Needs a GB300."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import generators as og
from oracle import hbaca as oh
from paper_1901_06101_gb300 import binding as B
from paper_1901_06101_gb300 import inputs
from tests import oracle_pool as opool
from tests.test_gpu_batched import levels_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return B.Context()


def _case(seed, m, n, nrhs):
    x, y = inputs.gaussian_pair(seed=seed, m=m, n=n)
    X = inputs.rhs(seed + 100, n, nrhs)
    return x, y, X


def _forward(ctx, x, y, h, X, L, d, eps, cap=256, flags=B.FLAG_TAPE):
    spec = B.gaussian(x, y, h)
    opts = B.make_opts(eps, d, L, seed=0, rank_cap=cap, leaf_rank_cap=cap, flags=flags)
    comp = B.compress(ctx, spec, opts)
    Y = B.apply(ctx, spec, comp, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    return spec, opts, comp, Y


def _oracle_loss(x, y, h, X, L, d, eps, traces, ranks=None):
    g = og.Gaussian(x, y, h)
    r = oh.hbaca(g, L, d, eps, seed=0, forced=traces, ranks=ranks)
    Ah = (r["U"] * r["s"][None, :]) @ r["V"]
    Y = Ah @ X
    return 0.5 * float(np.sum(Y * Y)), r


def test_tape_mode_leaves_the_result_unchanged(ctx):
    """A taped call accumulates the Jacobi rotations, an untaped one recovers
    the kept right vectors from X^H z = sigma w: the same ranks and, up to
    rounding, the same factors."""
    x, y, X = _case(11, 700, 650, 3)
    a = _forward(ctx, x, y, 0.7, X, 1, 8, 1e-8, flags=0)[2]
    b = _forward(ctx, x, y, 0.7, X, 1, 8, 1e-8, flags=B.FLAG_TAPE)[2]
    assert a.rank == b.rank
    assert float(torch.max(torch.abs(a.S - b.S))) <= 1e-13 * float(a.S[0])
    Aa = (a.U * a.S[None, :]) @ a.V
    Ab = (b.U * b.S[None, :]) @ b.V
    assert float(torch.linalg.norm(Aa - Ab)) <= 1e-12 * float(torch.linalg.norm(Aa))
    r = a.rank
    eye = torch.eye(r, dtype=a.U.dtype, device=a.U.device)
    assert float(torch.max(torch.abs(a.U.T @ a.U - eye))) <= 1e-12
    assert float(torch.max(torch.abs(a.V @ a.V.T - eye))) <= 1e-12


def test_apply_and_dX_match_dense_products(ctx):
    x, y, X = _case(12, 900, 800, 5)
    spec, opts, comp, Y = _forward(ctx, x, y, 0.7, X, 2, 8, 1e-8)
    Ah = (comp.U * comp.S[None, :]) @ comp.V
    Xt = torch.from_numpy(X).cuda()
    ref = Ah @ Xt
    assert float(torch.linalg.norm(Y - ref)) <= 1e-13 * float(torch.linalg.norm(ref))
    dY = torch.from_numpy(inputs.rhs(5, 900, 5)).cuda()
    dh, dx, dy, dX = B.apply_backward(ctx, spec, opts, comp, Xt, dY)
    refX = Ah.T @ dY
    assert float(torch.linalg.norm(dX - refX)) <= 1e-13 * float(torch.linalg.norm(refX))


@pytest.mark.parametrize("m,n,L,d", [(600, 520, 1, 8), (777, 513, 2, 8)])
def test_gradient_matches_frozen_pivot_finite_differences(ctx, m, n, L, d):
    eps, h, nrhs = 1e-8, 0.7, 4
    x, y, X = _case(21 + L, m, n, nrhs)
    spec, opts, comp, Y = _forward(ctx, x, y, h, X, L, d, eps)
    dh, dx, dy, _ = B.apply_backward(ctx, spec, opts, comp, torch.from_numpy(X).cuda(), Y, want_dX=False)
    dh = float(dh)
    dx = dx.cpu().numpy()
    dy = dy.cpu().numpy()
    nb = 1 << L
    traces = {leaf: B.read_leaf_trace(spec, opts, comp.ws, leaf) for leaf in range(nb * nb)}
    loss0, r0 = _oracle_loss(x, y, h, X, L, d, eps, traces)
    assert r0["r"] == comp.rank
    Ygpu = Y.cpu().numpy()
    assert abs(0.5 * float(np.sum(Ygpu * Ygpu)) - loss0) <= 1e-10 * loss0
    frozen = r0["ranks"]
    # d/dh by central differences, step 1e-6 h
    dlt = 1e-6 * h
    lp, rp = _oracle_loss(x, y, h + dlt, X, L, d, eps, traces, frozen)
    lm, rm = _oracle_loss(x, y, h - dlt, X, L, d, eps, traces, frozen)
    fd = (lp - lm) / (2 * dlt)
    assert abs(dh - fd) <= 1e-6 * abs(fd), (dh, fd)
    # directional derivatives in the point coordinates: 16 random directions
    rng = np.random.default_rng(7)
    for _ in range(16):
        px = rng.standard_normal(x.shape)
        py = rng.standard_normal(y.shape)
        t = 1e-6
        lp, _ = _oracle_loss(x + t * px, y + t * py, h, X, L, d, eps, traces, frozen)
        lm, _ = _oracle_loss(x - t * px, y - t * py, h, X, L, d, eps, traces, frozen)
        fd = (lp - lm) / (2 * t)
        an = float(np.sum(dx * px) + np.sum(dy * py))
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-12 * loss0), (an, fd)


def test_cfg5_structure_gradient_matches_frozen_pivot_finite_differences(ctx):
    """The differentiated workload's structure (d = 16, 8 x 8 leaves,
    eps = 1e-8, h = 0.7) at 4096^2, where the frozen-pivot oracle is
    affordable: dL/dh and two directional derivatives in the point
    coordinates against central finite differences (step 1e-6) of the oracle
    H-BACA with the GPU's pivots and the oracle's truncation ranks frozen,
    within 1e-6 relative."""
    eps, h, nrhs, L, d = 1e-8, 0.7, 8, 3, 16
    x, y, X = _case(61, 4096, 4096, nrhs)
    spec, opts, comp, Y = _forward(ctx, x, y, h, X, L, d, eps, cap=512)
    dh, dx, dy, _ = B.apply_backward(ctx, spec, opts, comp, torch.from_numpy(X).cuda(), Y, want_dX=False)
    dh = float(dh)
    dx = dx.cpu().numpy()
    dy = dy.cpu().numpy()
    traces = {leaf: B.read_leaf_trace(spec, opts, comp.ws, leaf) for leaf in range(64)}
    rng = np.random.default_rng(17)
    dirs = [(rng.standard_normal(x.shape), rng.standard_normal(y.shape)) for _ in range(2)]
    with opool.Pool() as pool:
        r0 = opool.hbaca(pool, og.Gaussian(x, y, h), L, d, eps, seed=0, forced=traces)
        assert r0["r"] == comp.rank
        A0 = (r0["U"] * r0["s"][None, :]) @ r0["V"]
        Y0 = A0 @ X
        loss0 = 0.5 * float(np.sum(Y0 * Y0))
        Ygpu = Y.cpu().numpy()
        assert abs(0.5 * float(np.sum(Ygpu * Ygpu)) - loss0) <= 1e-10 * loss0
        fr = r0["ranks"]
        dl, t = 1e-6 * h, 1e-6
        cases = [(x, y, h + dl, X, L, d, eps, traces, fr), (x, y, h - dl, X, L, d, eps, traces, fr)]
        for px, py in dirs:
            cases += [(x + t * px, y + t * py, h, X, L, d, eps, traces, fr),
                      (x - t * px, y - t * py, h, X, L, d, eps, traces, fr)]
        losses = opool.gaussian_losses(pool, cases)
    fd = (losses[0] - losses[1]) / (2 * dl)
    assert abs(dh - fd) <= 1e-6 * abs(fd), (dh, fd)
    for i, (px, py) in enumerate(dirs):
        fdd = (losses[2 + 2 * i] - losses[3 + 2 * i]) / (2 * t)
        an = float(np.sum(dx * px) + np.sum(dy * py))
        assert abs(an - fdd) <= 1e-6 * max(abs(fdd), 1e-12 * loss0), (i, an, fdd)


def test_gradient_close_to_dense_autograd(ctx):
    """The compressed map differs from A by O(eps): its gradient agrees with
    autograd through the dense matrix to well within 1e-6 (relative, in norm)."""
    eps, h, nrhs = 1e-10, 0.7, 4
    x, y, X = _case(31, 640, 600, nrhs)
    spec, opts, comp, Y = _forward(ctx, x, y, h, X, 1, 8, eps)
    dh, dx, dy, _ = B.apply_backward(ctx, spec, opts, comp, torch.from_numpy(X).cuda(), Y, want_dX=False)
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x, requires_grad=True)
    yt = torch.tensor(y, requires_grad=True)
    A = torch.exp(-torch.cdist(xt, yt) ** 2 / (2 * ht ** 2))
    loss = 0.5 * torch.sum((A @ torch.from_numpy(X)) ** 2)
    gh, gx, gy = torch.autograd.grad(loss, (ht, xt, yt))
    assert abs(float(dh) - float(gh)) <= 1e-6 * abs(float(gh))
    assert float(torch.linalg.norm(dx.cpu() - gx)) <= 1e-6 * float(torch.linalg.norm(gx))
    assert float(torch.linalg.norm(dy.cpu() - gy)) <= 1e-6 * float(torch.linalg.norm(gy))


def test_autograd_function(ctx):
    eps, h0, nrhs = 1e-8, 0.7, 2
    x, y, X = _case(41, 500, 450, nrhs)
    h = torch.tensor(h0, dtype=torch.float64, device="cuda", requires_grad=True)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    yt = torch.tensor(y, device="cuda", requires_grad=True)
    Xt = torch.tensor(X, device="cuda", requires_grad=True)
    Yh = B.gaussian_hbaca_apply(h, xt, yt, Xt, ctx, eps, 8, 1, rank_cap=256, leaf_rank_cap=256)
    loss = 0.5 * (Yh ** 2).sum()
    loss.backward()
    spec, opts, comp, Y = _forward(ctx, x, y, h0, X, 1, 8, eps)
    dh, dx, dy, dX = B.apply_backward(ctx, spec, opts, comp, torch.from_numpy(X).cuda(), Y)
    # two runs of the reverse pass differ only in the order of their atomic
    # sums, which the cancellation inside the LRID adjoint amplifies (seen:
    # 1.3e-9 relative); the gradient itself is checked against finite
    # differences at 1e-6 above
    assert abs(float(h.grad) - float(dh)) <= 1e-7 * abs(float(dh))
    assert float(torch.linalg.norm(xt.grad - dx)) <= 1e-7 * float(torch.linalg.norm(dx))
    assert float(torch.linalg.norm(yt.grad - dy)) <= 1e-7 * float(torch.linalg.norm(dy))
    assert float(torch.linalg.norm(Xt.grad - dX)) <= 1e-7 * float(torch.linalg.norm(dX))


def test_backward_refuses_untaped_workspace(ctx):
    x, y, X = _case(51, 300, 280, 2)
    spec, opts, comp, Y = _forward(ctx, x, y, 0.7, X, 1, 8, 1e-8, flags=0)
    tape_opts = B.make_opts(1e-8, 8, 1, seed=0, rank_cap=256, leaf_rank_cap=256, flags=B.FLAG_TAPE)
    with pytest.raises(B.HbacaError):
        B.apply_backward(ctx, spec, tape_opts, comp, torch.from_numpy(X).cuda(), Y)


def test_cfg5_full_size_gradient_against_dense_autograd(ctx):
    """The differentiated workload at full size (16384 x 16384, 8 x 8 leaves,
    d = 16, eps = 1e-8, 64 right-hand sides) against autograd through the
    dense kernel matrix on the GPU (torch, test-side reference only); the two
    differ by O(eps) relative."""
    m = n = 16384
    eps, h, nrhs = 1e-8, 0.7, 64
    x, y = inputs.gaussian_pair(seed=0, m=m, n=n)
    X = inputs.rhs(1, n, nrhs)
    spec, opts, comp, Y = _forward(ctx, x, y, h, X, 3, 16, eps, cap=512)
    Xt = torch.from_numpy(X).cuda()
    dh, dx, dy, dX = B.apply_backward(ctx, spec, opts, comp, Xt, Y)
    ht = torch.tensor(h, dtype=torch.float64, device="cuda", requires_grad=True)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    yt = torch.tensor(y, device="cuda", requires_grad=True)
    d2 = (xt * xt).sum(1)[:, None] + (yt * yt).sum(1)[None, :] - 2.0 * xt @ yt.T
    A = torch.exp(-d2 / (2 * ht ** 2))
    Yd = A @ Xt
    loss = 0.5 * torch.sum(Yd ** 2)
    gh, gx, gy = torch.autograd.grad(loss, (ht, xt, yt))
    assert float(torch.linalg.norm(Y - Yd)) <= 1e-6 * float(torch.linalg.norm(Yd))
    assert abs(float(dh) - float(gh)) <= 1e-5 * abs(float(gh)), (float(dh), float(gh))
    assert float(torch.linalg.norm(dx - gx)) <= 1e-5 * float(torch.linalg.norm(gx))
    assert float(torch.linalg.norm(dy - gy)) <= 1e-5 * float(torch.linalg.norm(gy))
    refX = A.detach().T @ Y
    assert float(torch.linalg.norm(dX - refX)) <= 1e-6 * float(torch.linalg.norm(refX))


def test_batched_backward_matches_dense_autograd_per_block(ctx):
    """One batched reverse pass over uneven Gaussian blocks (each with its own
    tree depth): every block's dL/dh, dL/dx, dL/dy against autograd through
    that block's dense kernel matrix (O(eps) apart), and dX exactly."""
    eps, nrhs = 1e-10, 3
    blocks = inputs.batched_blocks(seed=21, nblocks=6, lo=200, hi=700)
    specs = [B.gaussian(x, y, h) for (x, y, h) in blocks]
    opts = B.make_opts(eps, 8, -256, seed=0, rank_cap=256, leaf_rank_cap=256, flags=B.FLAG_TAPE)
    bt = B.Batch(ctx, specs, opts).run()
    torch.cuda.synchronize()
    Xs = [torch.from_numpy(inputs.rhs(300 + b, s.n, nrhs)).cuda() for b, s in enumerate(specs)]
    res = bt.results()
    Ys = [(r.U * r.S[None, :]) @ (r.V @ X) for r, X in zip(res, Xs)]
    dh, dx, dy, dX = B.apply_backward_batched(bt, Xs, Ys)
    for b, ((x, y, h), r, X, Y) in enumerate(zip(blocks, res, Xs, Ys)):
        Ah = (r.U * r.S[None, :]) @ r.V
        assert float(torch.linalg.norm(dX[b] - Ah.T @ Y)) <= 1e-12 * float(torch.linalg.norm(Ah.T @ Y))
        ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
        xt = torch.tensor(x, requires_grad=True)
        yt = torch.tensor(y, requires_grad=True)
        A = torch.exp(-torch.cdist(xt, yt) ** 2 / (2 * ht ** 2))
        loss = 0.5 * torch.sum((A @ X.cpu()) ** 2)
        gh, gx, gy = torch.autograd.grad(loss, (ht, xt, yt))
        # O(eps) apart; on the smoothest blocks (h ~ 5) the point gradients are
        # sums of nearly cancelling terms and the two agree to ~2e-6
        assert abs(float(dh[b]) - float(gh)) <= 1e-5 * abs(float(gh)) + 1e-12, (b, float(dh[b]), float(gh))
        assert float(torch.linalg.norm(dx[b].cpu() - gx)) <= 1e-5 * float(torch.linalg.norm(gx)) + 1e-12, b
        assert float(torch.linalg.norm(dy[b].cpu() - gy)) <= 1e-5 * float(torch.linalg.norm(gy)) + 1e-12, b
    # the reference proper for the smoothest block: central differences of the
    # oracle H-BACA with this block's pivots (batch index b) and ranks frozen
    b = max(range(len(blocks)), key=lambda i: blocks[i][2])
    x, y, h = blocks[b]
    L = levels_for(x.shape[0], y.shape[0], 256)
    nb = 1 << L
    traces = {leaf: B.read_leaf_trace_batched(specs, opts, bt.ws, b, leaf) for leaf in range(nb * nb)}
    Xn = Xs[b].cpu().numpy()

    def oloss(hh, ranks=None):
        r = oh.hbaca(og.Gaussian(x, y, hh), L, 8, eps, seed=0, batch_index=b, forced=traces, ranks=ranks)
        Yo = ((r["U"] * r["s"][None, :]) @ r["V"]) @ Xn
        return 0.5 * float(np.sum(Yo * Yo)), r

    _, r0 = oloss(h)
    dl = 1e-6 * h
    fd = (oloss(h + dl, r0["ranks"])[0] - oloss(h - dl, r0["ranks"])[0]) / (2 * dl)
    assert abs(float(dh[b]) - fd) <= 1e-6 * abs(fd), (float(dh[b]), fd)
