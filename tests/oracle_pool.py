"""Frozen-pivot oracle H-BACA over a process pool (test infrastructure).

The steps and their order are those of ``oracle.hbaca.hbaca`` with ``forced``
records: every leaf is the frozen-pivot replay of its recorded BACA run
(``oracle.baca.baca_replay``) followed by the SVD re-compression, then every
level's horizontal and vertical merges (Alg. 3).  Only the independent tasks
of one phase run side by side, in spawned processes with one BLAS thread
each, so large workloads finish in seconds; the arithmetic is the oracle's.
``test_oracle_pool_equals_serial_oracle`` checks that the result equals the
serial ``hbaca`` (to the rounding of BLAS products summed by another number
of threads).
"""
import os

import numpy as np

from oracle import generators as og


def leaf_generator(gen, r0, mr, c0, nc):
    """The generator of rows [r0, r0+mr) x columns [c0, c0+nc) of ``gen``,
    holding only that leaf's data (small enough to send to a worker)."""
    if isinstance(gen, og.Gaussian):
        return og.Gaussian(gen.x[r0:r0 + mr], gen.y[c0:c0 + nc], gen.h)
    if isinstance(gen, og.Helmholtz):
        return og.Helmholtz(gen.x[r0:r0 + mr], gen.y[c0:c0 + nc], gen.k)
    if isinstance(gen, og.SparseProduct):
        return og.SparseProduct(gen.P[r0:r0 + mr], gen.Q[:, c0:c0 + nc], gen.P2[r0:r0 + mr], gen.Q2[:, c0:c0 + nc])
    return og.Window(gen, r0, mr, c0, nc)


def _leaf(args):
    a, b, g, d, eps, seed, bid, rec, rank = args
    from oracle import baca as ob
    if rec is None:
        res = ob.baca(g, d, eps, seed=seed, bid=bid)
        recs = None
    else:
        res = ob.baca_replay(g, d, eps, rec["trace"], seed=seed, bid=bid, stop=rec.get("stop", "converged"))
        recs = res["recs"]
    U, s, V = ob.recompress(res["U"], res["V"], eps, rank)
    return a, b, U, s, V, res["r"], recs


def _merge(args):
    kind, U1, s1, V1, U2, s2, V2, eps, rank = args
    from oracle import hbaca as oh
    f = oh.horizontal_merge if kind == "h" else oh.vertical_merge
    return f(U1, s1, V1, U2, s2, V2, eps, rank)


class Pool:
    """Spawned worker processes with one BLAS thread each."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = max(1, min(len(os.sched_getaffinity(0)), procs or 64))
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def map(self, fn, jobs):
        return self.pool.map(fn, jobs, chunksize=1)

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hbaca(pool, gen, L, d, eps, seed=0, batch_index=0, forced=None, ranks=None):
    """oracle.hbaca.hbaca(gen, L, d, eps, seed, batch_index, forced=forced,
    ranks=ranks) with the leaves of a level, and the merges of a level, spread
    over ``pool``.  Returns U, s, V, r, the truncation ranks taken (same keys
    as the serial oracle), the leaf BACA ranks and the replay records."""
    from oracle import hbaca as oh
    from oracle import sampler as osamp

    def rk(key):
        return None if ranks is None else ranks.get(key)
    rows = oh.tree_levels(gen.m, L)
    cols = oh.tree_levels(gen.n, L)
    nbc = len(cols[0])
    jobs = []
    for a, (r0, mr) in enumerate(rows[0]):
        for b, (c0, nc) in enumerate(cols[0]):
            leaf = a * nbc + b
            rec = forced.get(leaf) if forced is not None else None
            jobs.append((a, b, leaf_generator(gen, r0, mr, c0, nc), d, eps, seed,
                         osamp.block_id(batch_index, a, b), rec, rk(("full", 0, a, b))))
    taken, blocks, leaf_rank, leaf_recs = {}, {}, {}, {}
    for a, b, U, s, V, rb, recs in pool.map(_leaf, jobs):
        blocks[(a, b)] = (U, s, V)
        taken[("full", 0, a, b)] = len(s)
        leaf_rank[(a, b)] = rb
        leaf_recs[(a, b)] = recs
    for l in range(1, L + 1):
        keys = [(a, b) for a in range(len(rows[l - 1])) for b in range(len(cols[l]))]
        res = pool.map(_merge, [("h",) + blocks[(a, 2 * b)] + blocks[(a, 2 * b + 1)] + (eps, rk(("half", l, a, b)))
                                for (a, b) in keys])
        half = dict(zip(keys, res))
        for key, v in half.items():
            taken[("half", l) + key] = len(v[1])
        keys = [(a, b) for a in range(len(rows[l])) for b in range(len(cols[l]))]
        res = pool.map(_merge, [("v",) + half[(2 * a, b)] + half[(2 * a + 1, b)] + (eps, rk(("full", l, a, b)))
                                for (a, b) in keys])
        blocks = dict(zip(keys, res))
        for key, v in blocks.items():
            taken[("full", l) + key] = len(v[1])
    U, s, V = blocks[(0, 0)]
    return dict(U=U, s=s, V=V, r=len(s), ranks=taken, leaf_rank=leaf_rank, leaf_recs=leaf_recs)


def _loss(args):
    """0.5 ||A_hat X||^2 of the serial frozen-pivot oracle H-BACA of a
    Gaussian kernel matrix (one finite-difference evaluation)."""
    x, y, h, X, L, d, eps, forced, ranks = args
    from oracle import hbaca as oh
    r = oh.hbaca(og.Gaussian(x, y, h), L, d, eps, seed=0, forced=forced, ranks=ranks)
    Y = ((r["U"] * r["s"][None, :]) @ r["V"]) @ X
    return 0.5 * float(np.sum(Y * Y))


def gaussian_losses(pool, cases):
    """_loss of every (x, y, h, X, L, d, eps, forced, ranks) case, in
    parallel."""
    return pool.map(_loss, cases)
