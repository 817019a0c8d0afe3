"""Host-side planning (no GPU): the workspace regions of a plan are disjoint
and inside the total, and the leaf BACA cluster size follows the rounds rule
(persistent clusters of c CTAs take the leaves in ceil(leaves / (SMs / c))
rounds of a leaf time that falls as 1 / c; ties to the smaller c).  The
planner assumes 152 SMs when no device is present."""
import numpy as np
import pytest

from paper_1901_06101_gb300 import binding as B

REGIONS = ["status", "queue", "desc", "uar", "var", "qr", "tau", "core", "ord", "full_u", "full_s", "full_v",
           "half_u", "half_s", "half_v", "cscr", "rscr", "gscr", "tape_int", "tape_dbl", "jlist", "xpart", "xcnt"]


def _plan(m, n, L, d=16, cluster=0, cplx=True, flags=0):
    kind, dt = (B.GEN_HELMHOLTZ, B.C128) if cplx else (B.GEN_GAUSSIAN, B.F64)
    # the planner never dereferences the point arrays: any non-null address will do
    g = B.Gen(kind=kind, dtype=dt, m=m, n=n, x=4096, y=8192, dim=3, k=4 * np.pi, h=1.0)
    spec = B.GenSpec(g, ())
    opts = B.make_opts(1e-4, d, L, seed=1, rank_cap=256, leaf_rank_cap=256, cluster=cluster, flags=flags)
    return B.plan_json(spec, opts)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("libhbaca.so not built")


@pytest.mark.parametrize("flags", [0, B.FLAG_TAPE])
def test_regions_disjoint_and_inside_the_workspace(flags):
    j = _plan(20000, 20000, 4, flags=flags)
    spans = sorted((j[r][0], j[r][0] + max(j[r][1], 1), r) for r in REGIONS)
    for (a0, a1, ra), (b0, b1, rb) in zip(spans, spans[1:]):
        assert a1 <= b0, (ra, rb)
    assert spans[-1][1] <= j["total"]
    assert all(j[r][0] % 256 == 0 for r in REGIONS)


def rounds_rule(leaves, mmax, sms=152):
    best, pick = None, 1
    for c in (1, 2, 4, 8):
        if c > 1 and -(-mmax // c) < 16:
            break
        clusters = max(1, sms // c)
        cost = -(-leaves // clusters) / c
        if best is None or cost < best * (1 - 1e-9):
            best, pick = cost, c
    return pick


@pytest.mark.parametrize("m,L,expect", [(20000, 4, 4), (2000, 2, 8), (50000, 5, 4), (40000, 6, 1)])
def test_baca_cluster_follows_the_rounds_rule(m, L, expect):
    j = _plan(m, m, L)
    leaves, mmax = 4 ** L, -(-m // 2 ** L)
    assert rounds_rule(leaves, mmax) == expect
    assert j["baca_cluster"] == expect


def test_explicit_cluster_size_is_kept():
    assert _plan(20000, 20000, 4, cluster=2)["baca_cluster"] == 2


@pytest.mark.parametrize("L", [0, 2, 4])
def test_frobenius_budget_per_task(L):
    """HBACA_FLAG_FROB: every leaf re-compression and merge task carries the
    divisor 2L + 1 of its Frobenius budget eps / sqrt(2L + 1); without the
    flag every task keeps the eps-rank (0)."""
    m = 20000 if L else 1200
    plain = _plan(m, m, L)
    frob = _plan(m, m, L, flags=B.FLAG_FROB)
    for j, want in ((plain, 0), (frob, 2 * L + 1)):
        tasks = [t for st in j["stages"] for t in st["tasks"]]
        # 4^L leaves; per level l, 2 * 4^(L-l) horizontal and 4^(L-l) vertical merges
        assert len(tasks) == 4 ** L + sum(3 * 4 ** (L - l) for l in range(1, L + 1))
        assert all(t["trunc"] == want for t in tasks)
    nstages = 1 + 2 * L
    assert len(frob["stages"]) == nstages


def _size_error(kind, dtype, flags=0, eps=1e-4, d=16, L=2, **fields):
    g = B.Gen(kind=kind, dtype=dtype, m=2000, n=1800, x=4096, y=8192, dim=3, **fields)
    opts = B.make_opts(eps, d, L, seed=1, rank_cap=128, leaf_rank_cap=128, flags=flags)
    try:
        B.workspace_size(g, opts)
    except B.HbacaError as e:
        return str(e)
    return None


@pytest.mark.parametrize("case", [
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=float("nan")),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=float("inf")),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=0.0),
    dict(kind=B.GEN_HELMHOLTZ, dtype=B.C128, k=float("nan")),
    dict(kind=B.GEN_HELMHOLTZ, dtype=B.C128, k=float("inf")),
    dict(kind=B.GEN_POLYNOMIAL, dtype=B.F64, h=float("inf")),
    dict(kind=B.GEN_HANKEL2D, dtype=B.C128, k=float("inf")),
    dict(kind=B.GEN_HANKEL2D, dtype=B.C128, k=-1.0),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.C128, h=1.0),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=1.0, eps=float("nan")),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=1.0, eps=1.0),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=1.0, d=33),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=1.0, L=11),
    dict(kind=B.GEN_GAUSSIAN, dtype=B.F64, h=1.0, flags=64),
])
def test_invalid_parameters_are_refused_when_planning(case):
    """Faults injected on the host: a NaN or infinite generator parameter, a
    wrong dtype, tolerance, block size or depth, or an unknown option flag is
    refused (HBACA_INVALID_ARG with a message) before any launch."""
    msg = _size_error(**case)
    assert msg, case


def test_valid_parameters_plan():
    assert _size_error(B.GEN_GAUSSIAN, B.F64, h=0.7) is None
    assert _size_error(B.GEN_HELMHOLTZ, B.C128, k=4 * np.pi, flags=B.FLAG_FROB | B.FLAG_TAPE) is None
