"""The pooled frozen-pivot oracle driver (tests/oracle_pool.py) runs the
serial oracle's steps: the same ranks and, up to the rounding of BLAS
products summed by another number of threads, the same factors, free and
with forced pivot records, with frozen truncation ranks."""
import numpy as np

from oracle import baca as ob
from oracle import generators as og
from oracle import hbaca as oh
from oracle import sampler as osamp
from paper_1901_06101_gb300 import inputs
from tests import oracle_pool as opool


def _records(gen, L, d, eps, seed):
    """Pivot records of a free oracle run of every leaf, in the form the GPU
    trace reader returns (I, J, jbar, dk per iteration, the stop reason)."""
    rows = oh.tree_levels(gen.m, L)[0]
    cols = oh.tree_levels(gen.n, L)[0]
    out = {}
    for a, (r0, mr) in enumerate(rows):
        for b, (c0, nc) in enumerate(cols):
            res = ob.baca(og.Window(gen, r0, mr, c0, nc), d, eps, seed=seed, bid=osamp.block_id(0, a, b))
            out[a * len(cols) + b] = {"stop": res["stop"],
                                      "trace": [dict(I=t["I"], J=t["J"], jbar=t["jbar"], dk=t["dk"])
                                                for t in res["trace"]]}
    return out


def _same(got, want):
    np.testing.assert_allclose(got["s"], want["s"], rtol=0, atol=1e-13 * want["s"][0])
    Ag = (got["U"] * got["s"]) @ got["V"]
    Aw = (want["U"] * want["s"]) @ want["V"]
    assert np.linalg.norm(Ag - Aw) <= 1e-12 * np.linalg.norm(Aw)


def test_oracle_pool_equals_serial_oracle():
    x, y = inputs.gaussian_pair(seed=4, m=700, n=610)
    g = og.Gaussian(x, y, 0.8)
    rec = _records(g, 2, 8, 1e-8, 3)
    with opool.Pool(4) as pool:
        for forced in (None, rec):
            want = oh.hbaca(g, 2, 8, 1e-8, seed=3, forced=forced)
            got = opool.hbaca(pool, g, 2, 8, 1e-8, seed=3, forced=forced)
            assert got["r"] == want["r"] and got["ranks"] == want["ranks"]
            _same(got, want)
        frozen = {k: max(1, v - 1) for k, v in want["ranks"].items()}
        want = oh.hbaca(g, 2, 8, 1e-8, seed=3, forced=rec, ranks=frozen)
        got = opool.hbaca(pool, g, 2, 8, 1e-8, seed=3, forced=rec, ranks=frozen)
        assert got["ranks"] == want["ranks"]
        _same(got, want)


def test_leaf_generator_slices_match_windows():
    sp = inputs.sparse_product(seed=5, m=300, n=280, K=7, density=0.05)
    g = og.SparseProduct(sp.dense_P(), sp.dense_Q(), sp.P2, sp.Q2)
    xs, ys = inputs.sphere_pair(seed=2, m=90, n=80)
    for gen in (g, og.Helmholtz(xs, ys, 3.0), og.Gaussian(xs, ys, 0.5)):
        w = og.Window(gen, 11, 40, 7, 33)
        s = opool.leaf_generator(gen, 11, 40, 7, 33)
        I, J = np.arange(40), np.arange(33)
        assert np.array_equal(w(I, J), s(I, J))
