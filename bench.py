"""Benchmark of the H-BACA hot path on GB300.

Workload (one "step"): H-BACA compression of the Helmholtz kernel matrix
A(i, j) = exp(i k r) / r, complex128, m = n = 20000, points uniform on two unit
spheres centred 3 apart, k = 4 pi, seed 1; block size d = 16, 16 x 16 leaves
(L = 4), eps = 1e-4.  Inputs are synthetic (the paper's data sets are not
available) and resident in HBM when the timed region starts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  value = matrix entries generated per second
by the leaf BACA over the whole job; ms_per_step = device time of one
compression (CUDA events on the launching stream).  Between timed steps L2 is
flushed by writing a 512 MiB buffer.  With N > 1 (torchrun) every rank
compresses its own copy of the workload (the path has no exchange between
independent problems): weak scaling, replicas.

The same line carries compact results of the other workloads (rank 0, N = 1):
cfg1 (Gaussian 2000^2), cfg3 (coherent sparse product 50000^2, with plain ACA
beside it), cfg4 (4096 batched Gaussian blocks against the per-block loop) and
cfg5 (differentiated Gaussian 16384^2: backward / forward time).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H-BACA compress ms & entries/s at stated ε; batched vs per-block; bwd/fwd"
WORKLOADS = {
    # the benchmark configuration
    "helmholtz20000": dict(workload="helmholtz_c128_20000_d16_L4_eps1e-4", kernel="helmholtz exp(ikr)/r",
                           m=20000, n=20000, k=4 * np.pi, d=16, levels=4, eps=1e-4, seed=1,
                           rank_cap=256, leaf_rank_cap=256),
    # the same kernel at 8000^2 with 8 x 8 leaves of 1000^2: small enough for
    # multi-pass profiler captures, larger than L2
    "helmholtz8000": dict(workload="helmholtz_c128_8000_d16_L3_eps1e-4", kernel="helmholtz exp(ikr)/r",
                          m=8000, n=8000, k=4 * np.pi, d=16, levels=3, eps=1e-4, seed=1,
                          rank_cap=256, leaf_rank_cap=256),
    # 4096 independent admissible Gaussian-kernel blocks of uneven sizes
    # (m, n log-uniform in [64, 2048], h log-uniform in [0.1, 10], seed 3),
    # leaves of at most 512 rows and columns: one batched call against the
    # plain loop of one call per block at the same eps
    # differentiated H-BACA: Gaussian kernel between 16384 points in [0,1]^3
    # and 16384 in [2,3]x[0,1]^2, h = 0.7, eps = 1e-8, d = 16, 8 x 8 leaves;
    # forward = taped compression + y = U(S(VX)) for 64 N(0,1) right-hand
    # sides, backward = dL/dh, dL/dx, dL/dy, dL/dX of L = 0.5 ||y||^2
    "grad16384": dict(workload="gaussian_f64_16384_d16_L3_eps1e-8_nrhs64_grad", kernel="gaussian",
                      m=16384, n=16384, h=0.7, d=16, levels=3, eps=1e-8, seed=0, nrhs=64,
                      rank_cap=512, leaf_rank_cap=384),
    # the differentiated workload batched: 256 Gaussian blocks, m, n
    # log-uniform in [256, 2048], h = 0.7, eps = 1e-8, d = 16, leaves of at most
    # 256 rows and columns, 64 right-hand sides per block
    "gradbatch256": dict(workload="gaussian_f64_256_blocks_256-2048_d16_leaf256_eps1e-8_nrhs64_grad",
                         kernel="gaussian", nblocks=256, h=0.7, d=16, levels=-256, eps=1e-8, seed=5, nrhs=64,
                         rank_cap=256, leaf_rank_cap=256),
    "batched4096": dict(workload="gaussian_f64_4096_blocks_64-2048_d8_leaf512_eps1e-8", kernel="gaussian",
                        nblocks=4096, d=8, levels=-512, eps=1e-8, seed=3, rank_cap=256, leaf_rank_cap=256),
}
WORKLOAD = WORKLOADS["helmholtz20000"]
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x DFMA/clk/SM x flop/FMA x max SM clock
# DRAM bytes (read + write) per launch of the current kernels on the default
# workload, averaged over one compression's launches (ncu dram__bytes_read.sum
# + dram__bytes_write.sum); None where no capture of the current kernel exists
TRAFFIC_PER_LAUNCH = {"helmholtz20000": {"jacobi_kernel": 15.67e6, "qr_kernel": 33.67e9, "qapply_kernel": 16.92e9,
                                         "baca_leaf_kernel": 11.56e9}}


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json beside this
    file), or None when the file is absent."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


EXTRA_FLAGS = 0  # option flags added to every call (--single-cluster)


def mk_opts(*a, flags=0, **kw):
    from paper_1901_06101_gb300 import binding as B
    return B.make_opts(*a, flags=flags | EXTRA_FLAGS, **kw)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", default="helmholtz20000", choices=sorted(WORKLOADS))
    ap.add_argument("--nblocks", type=int, default=None, help="batched workload: first N blocks only")
    ap.add_argument("--no-loop", action="store_true", help="batched workload: skip the per-block loop")
    ap.add_argument("--single-cluster", action="store_true",
                    help="one cluster per matrix in QR / Q application (for profilers that serialise launches)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads' keys (cfg1, cfg3-5)")
    ap.add_argument("--loop-blocks", type=int, default=256,
                    help="cfg4: blocks timed by the per-block loop (scaled to all blocks)")
    return ap.parse_args()


# ------------------------------------------------------------------ work accounting
def leaf_spans(n, L):
    """Leaves of the L-level index tree on [0, n) (first child ceil(s/2))."""
    spans = [(0, n)]
    for _ in range(L):
        nxt = []
        for s0, sz in spans:
            a = (sz + 1) // 2
            nxt += [(s0, a), (s0 + a, sz - a)]
        spans = nxt
    return spans


# ------------------------------------------------------------------ ranks
def max_over_ranks(v, world, device="cpu"):
    """The largest value of one float over all ranks: the slowest replica sets
    the job's time.  device: where the reduction tensor lives (a CUDA device
    for NCCL, "cpu" for gloo)."""
    if world <= 1:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_max, world):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank, timed by the slowest of them (weak scaling)."""
    return world * units_per_rank / seconds_max


def jacobi_accounting(ws, plan, complex_, accumulates=False):
    """Algorithmic FP64 flops of the Jacobi SVD launches of one compression,
    from the per-task records the kernel leaves (sizes, sweeps, rotations):
    every sweep forms the squared norm of each of the nc columns once and the
    inner product of each of the nc (nc - 1) / 2 column pairs over the mr rows
    of the core (the norms are carried through the rotations), and every
    applied rotation updates both columns of the core (mr rows), and of the
    accumulated rotation (nc rows) when the call is taped (``accumulates``).
    Per element: norm 4 flops (complex) / 2 (real), inner product 8 / 2,
    rotation 18 / 7."""
    import torch
    fn, fd, fr = (4.0, 8.0, 18.0) if complex_ else (2.0, 2.0, 7.0)
    total = 0.0
    for st in plan["stages"]:
        nt = st["ntasks"]
        d = ws[st["dims"]: st["dims"] + 32 * nt].view(torch.int32).view(nt, 8).cpu().numpy()
        for k, kra, krb, s_, sweeps, nout, rot, _ in d:
            ncm = krb if st["kind"] == 0 else k
            mr, nc = int(ncm), int(min(kra, ncm))
            if nc < 2:
                continue
            nsw = min(int(sweeps) + 1, 40)
            total += nsw * (nc * mr * fn + nc * (nc - 1) / 2 * mr * fd) + float(rot) * (mr + (nc if accumulates else 0)) * fr
    return total


def jacobi_stage_stats(ws, plan):
    """Per stage of one compression: tasks, mean core columns and the mean and
    largest number of Jacobi sweeps (from the per-task records)."""
    import torch
    out = []
    for st in plan["stages"]:
        nt = st["ntasks"]
        d = ws[st["dims"]: st["dims"] + 32 * nt].view(torch.int32).view(nt, 8).cpu().numpy()
        ncm = d[:, 2] if st["kind"] == 0 else d[:, 0]
        nc = np.minimum(d[:, 1], ncm)
        sw = np.minimum(d[:, 4] + 1, 40)
        out.append({"tasks": int(nt), "cols": round(float(nc.mean()), 1), "sweeps_mean": round(float(sw.mean()), 2),
                    "sweeps_max": int(sw.max())})
    return out


def leaf_accounting(traces, leaf_sizes, d, complex_):
    """Entries generated and algorithmic FP64 flops of the leaf BACA (Alg. 2)
    from the per-leaf pivot records: per iteration with running rank r,
    C panel m r dJ MACs, R panel dI n r, QRCP of C^t / R (3 MACs per
    candidate component per step), V_k = T^-1 Q^H R n dk dI, Gram norms
    (m + n)(r + dk) dk.  A complex MAC is 8 real flops, a real one 2."""
    entries = 0
    macs = 0
    for tr, (m, n) in zip(traces, leaf_sizes):
        r = 0
        kept_r = 0
        kept_c = 0
        for rec in tr["trace"]:
            dI, dJ, dk = len(rec["I"]), len(rec["J"]), rec["dk"]
            entries += m * dJ + dI * n
            macs += m * r * dJ + dI * n * r
            macs += sum(3 * (dJ - t) * (m - kept_r) for t in range(dI))
            macs += sum(3 * (dI - t) * max(n - kept_c - dJ, 0) for t in range(min(d, dI)))
            macs += n * dk * dI + (m + n) * (r + dk) * dk
            r += dk
            kept_r += dk
            kept_c += dk
    return entries, macs * (8 if complex_ else 2)


def task_dims(ws, plan):
    """Per stage: (kind, device-written task sizes (ntasks x 8 ints: k, kra,
    krb, s, sweeps, nout, rotations, pad), rows of the stacked QR operand per
    task, and rows of the second QR operand (leaf tasks; 0 for merges))."""
    import torch
    out = []
    for st in plan["stages"]:
        nt = st["ntasks"]
        d = ws[st["dims"]: st["dims"] + 32 * nt].view(torch.int32).view(nt, 8).cpu().numpy()
        rows = np.array([t["rows_a"] for t in st["tasks"]], np.int64)
        rows_b = np.array([t["rows_b"] if st["kind"] == 0 else 0 for t in st["tasks"]], np.int64)
        out.append((st["kind"], d, rows, rows_b))
    return out


def qr_flops(m, k):
    """Householder QR of an m x k matrix (LAPACK geqrf count): the reflector of
    column j (m - j rows) applied to the k - j - 1 columns after it, two
    flops per entry for the inner products and two for the update."""
    m = np.asarray(m, np.float64)
    k = np.minimum(np.asarray(k, np.float64), m)
    return 2.0 * m * k ** 2 - 2.0 * k ** 3 / 3.0


def qapply_flops(m, k, s):
    """Q [Z; 0] for the Q of k Householder reflectors of m rows applied to s
    columns (LAPACK ormqr count): reflector j touches m - j rows of every
    column, two flops per entry for the inner product and two for the update."""
    m = np.asarray(m, np.float64)
    k = np.asarray(k, np.float64)
    s = np.asarray(s, np.float64)
    return 4.0 * m * k * s - 2.0 * k ** 2 * s


def jacobi_flops_8d(dims, complex_):
    """Algorithmic flops of the core SVDs by the work count of the plan's
    measurement section: 20 r^3 per leaf re-compression core (r = its
    columns) and 20 (2 s)^3 per merge core (2 s = r1 + r2 stacked columns),
    four times that for complex data."""
    tot = 0.0
    for kind, d, _, _ in dims:
        ncm = d[:, 2] if kind == 0 else d[:, 0]
        nc = np.minimum(d[:, 1], ncm).astype(np.float64)
        tot += float(np.sum(20.0 * nc ** 3))
    return tot * (4.0 if complex_ else 1.0)


def whole_flops_8d(traces, leaf_sizes, d, dims, complex_):
    """Algorithmic flops of one whole compression by the same work count:
    per leaf (m, n, BACA rank r) (m + n) 2 r^2 (updates and norms) +
    2 d r (m + n) (pivot QRCPs) + 2 d r n (LRID) + 4 (m + n) r^2 + 20 r^3
    (re-compression); per merge (stacked side of `rows`, output rank s)
    12 rows s^2 + 20 (2 s)^3; four times that for complex data."""
    tot = 0.0
    for tr, (m, n) in zip(traces, leaf_sizes):
        r = float(tr["rank_baca"])
        tot += (m + n) * 2 * r * r + 2 * d * r * (m + n) + 2 * d * r * n + 4 * (m + n) * r * r + 20 * r ** 3
    for kind, dd, rows, _ in dims:
        if kind == 0:
            continue
        sv = dd[:, 3].astype(np.float64)
        tot += float(np.sum(12.0 * rows * sv ** 2 + 20.0 * (2 * sv) ** 3))
    return tot * (4.0 if complex_ else 1.0)


def dense_flops(dims, complex_):
    """(QR flops, Q-application flops) of one compression's re-compression and
    merge stages: a leaf task factors both of its BACA factors (rows_a x k
    and rows_b x k) and applies both Qs to its nout output columns; a merge
    factors and applies the stacked side only (the block-diagonal side is a
    plain product).  Four times that for complex data."""
    qr = qa = 0.0
    for kind, d, rows, rows_b in dims:
        k = d[:, 0].astype(np.float64)
        nout = d[:, 5].astype(np.float64)
        qr += float(np.sum(qr_flops(rows, k)))
        qa += float(np.sum(qapply_flops(rows, d[:, 1], nout)))
        if kind == 0:
            qr += float(np.sum(qr_flops(rows_b, k)))
            qa += float(np.sum(qapply_flops(rows_b, d[:, 2], nout)))
    f = 4.0 if complex_ else 1.0
    return qr * f, qa * f


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ CPU oracle baseline
# The oracle's own functions (BACA + re-compression per leaf, Alg. 2 and Sec.
# 3.2; the horizontal and vertical merges of Alg. 3) in the order of
# oracle.hbaca.hbaca, with the independent tasks of each phase spread over
# spawned processes of one BLAS thread each.
def _oracle_leaf(args):
    x, y, k, d, eps, seed, a, b = args
    from oracle import baca as ob
    from oracle import generators as og
    from oracle import sampler as osamp
    t0 = time.perf_counter()
    g = og.Helmholtz(x, y, k)  # the leaf's own rows / columns of the matrix
    res = ob.baca(g, d, eps, seed=seed, bid=osamp.block_id(0, a, b))
    U, s, V = ob.recompress(res["U"], res["V"], eps)
    entries = sum(g.m * len(t["J"]) + len(t["I"]) * g.n for t in res["trace"])
    return a, b, U, s, V, entries, time.perf_counter() - t0


def _oracle_merge(args):
    kind, U1, s1, V1, U2, s2, V2, eps = args
    from oracle import hbaca as oh
    f = oh.horizontal_merge if kind == "h" else oh.vertical_merge
    return f(U1, s1, V1, U2, s2, V2, eps)


def _warm(_):
    import oracle.hbaca  # noqa: F401
    return 0


class OraclePool:
    """A pool of spawned processes with one BLAS thread each (the thread
    limits are in the environment the children start with, so their numpy
    reads them on import)."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0))
        self.procs = max(1, min(cores, procs or cores))
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs)
            self.pool.map(_warm, range(self.procs))  # interpreter start-up outside any timing
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def close(self):
        self.pool.terminate()
        self.pool.join()


def oracle_hbaca_pool(op, x, y, k, L, d, eps, seed):
    """Oracle H-BACA of the Helmholtz matrix (x, y, k) with 4^L leaves on the
    pool: all leaves, then every merge level.  Returns (entries generated by
    the leaf BACA, wall seconds, final rank)."""
    rows = leaf_spans(x.shape[0], L)
    cols = leaf_spans(y.shape[0], L)
    nb = 1 << L
    t0 = time.perf_counter()
    jobs = [(x[rows[a][0]:rows[a][0] + rows[a][1]], y[cols[b][0]:cols[b][0] + cols[b][1]], k, d, eps, seed, a, b)
            for a in range(nb) for b in range(nb)]
    blocks, entries = {}, 0
    for a, b, U, s, V, e, _ in op.pool.imap_unordered(_oracle_leaf, jobs):
        blocks[(a, b)] = (U, s, V)
        entries += e
    nr = nc = nb
    while nr > 1:
        half = op.pool.map(_oracle_merge, [("h",) + blocks[(a, 2 * c)] + blocks[(a, 2 * c + 1)] + (eps,)
                                           for a in range(nr) for c in range(nc // 2)])
        nc //= 2
        hb = {(a, c): half[a * nc + c] for a in range(nr) for c in range(nc)}
        full = op.pool.map(_oracle_merge, [("v",) + hb[(2 * a, c)] + hb[(2 * a + 1, c)] + (eps,)
                                           for a in range(nr // 2) for c in range(nc)])
        nr //= 2
        blocks = {(a, c): full[a * nc + c] for a in range(nr) for c in range(nc)}
    return entries, time.perf_counter() - t0, len(blocks[(0, 0)][1])


def oracle_baseline(x, y, cfg, op=None):
    """The oracle on the whole benchmark compression (every leaf and every
    merge).  Returns the cpu_baseline record."""
    own = op is None
    op = op or OraclePool()
    try:
        entries, dt, rank = oracle_hbaca_pool(op, x, y, cfg["k"], cfg["levels"], cfg["d"], cfg["eps"], cfg["seed"])
    finally:
        if own:
            op.close()
    desc = ("oracle H-BACA of the whole workload: BACA + SVD re-compression of all %d leaves (Alg. 2, Sec. 3.2) and "
            "every merge level (Alg. 3), %d spawned processes x 1 BLAS thread; oracle rank %d"
            % (4 ** cfg["levels"], op.procs, rank))
    return {"value": entries / dt, "unit": "entries/s", "cores": op.procs, "kind": "oracle", "sample": desc,
            "seconds": dt}


# ------------------------------------------------------------------ GPU arm
def _timed_calls(fn, steps, warmup, flush, stream):
    """Run fn warmup + steps times; the last `steps` are timed with CUDA
    events on `stream`, L2 flushed before each.  Returns the mean ms and the
    last result."""
    import torch
    out = None
    for _ in range(warmup):
        out = fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms)), out


def _leaf_records(B, spec, opts, ws, m, n, L):
    nb = 1 << L
    rows, cols = leaf_spans(m, L), leaf_spans(n, L)
    traces, sizes = [], []
    for leaf in range(nb * nb):
        traces.append(B.read_leaf_trace(spec, opts, ws, leaf))
        a, b = divmod(leaf, nb)
        sizes.append((rows[a][1], cols[b][1]))
    return traces, sizes


def measure_single(B, ctx, spec, opts, cap, m, n, L, d, complex_, steps, warmup, flush, stream, dev):
    """Time hbaca_compress on one matrix and account its work.  Returns a
    dict: ms, entries, flops (whole compression and Jacobi, by the work
    count of the measurement section; leaf BACA by its own count), kernel
    times of one profiled call, phases, rank."""
    import torch
    dt = torch.complex128 if complex_ else torch.float64
    ws = torch.empty(B.workspace_size(spec.gen, opts), dtype=torch.uint8, device=dev)
    out = (torch.empty((cap, m), dtype=dt, device=dev), torch.empty(cap, dtype=torch.float64, device=dev),
           torch.empty((cap, n), dtype=dt, device=dev))
    ms, res = _timed_calls(lambda: B.compress(ctx, spec, opts, ws=ws, out=out), steps, warmup, flush, stream)
    traces, sizes = _leaf_records(B, spec, opts, ws, m, n, L)
    entries, leaf_flops = leaf_accounting(traces, sizes, d, complex_)
    popts = B.make_opts(opts.eps, opts.d, opts.levels, seed=opts.seed, rank_cap=opts.rank_cap,
                        leaf_rank_cap=opts.leaf_rank_cap, flags=opts.flags | B.FLAG_PROFILE, cluster=opts.cluster)
    res = B.compress(ctx, spec, popts, ws=ws, out=out)
    torch.cuda.synchronize(dev)
    (tb, tr, tm, tt), launches = B.phase_times(ctx)
    kt = B.kernel_times(ctx)
    plan = B.plan_json(spec, popts)
    dims = task_dims(ws, plan)
    return dict(ms=ms, res=res, ws=ws, out=out, entries=entries, leaf_flops=leaf_flops, traces=traces,
                whole_flops=whole_flops_8d(traces, sizes, d, dims, complex_),
                jacobi_flops=jacobi_flops_8d(dims, complex_),
                jacobi_own_flops=jacobi_accounting(ws, plan, complex_), jacobi_stages=jacobi_stage_stats(ws, plan),
                ktimes=kt, phases={"leaf_baca_ms": tb, "leaf_recompression_ms": tr, "merge_ms": tm},
                launches=launches, rank=res.rank)


def roofline_of(kname, flops, ktimes, traffic=None, note=None):
    kms, kl = ktimes[kname]
    ach = flops / (kms / 1e3) / 1e12
    r = {"bound": "alu", "kernel": kname, "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
         "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic, "flops_per_launch": flops / max(kl, 1),
         "ms_per_launch": kms / max(kl, 1), "launches": kl}
    if note:
        r["peak_note"] = note
    hbm = measured_hbm_gbs()
    if traffic and hbm:
        # the same launches against the memory roofline: DRAM bytes per launch
        # (ncu) over the event-timed launch time, of the measured copy bandwidth
        gbs = traffic / (r["ms_per_launch"] / 1e3) / 1e9
        r["dram"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    return r


def run_ours(args, rank, world):
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs

    cfg = WORKLOAD
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    x, y = inputs.sphere_pair(seed=cfg["seed"], m=cfg["m"], n=cfg["n"])
    ctx = B.Context()
    spec = B.helmholtz(x, y, cfg["k"])
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=cfg["seed"], rank_cap=cfg["rank_cap"],
                   leaf_rank_cap=cfg["leaf_rank_cap"], flags=B.FLAG_PROFILE)
    ws = torch.empty(B.workspace_size(spec.gen, opts), dtype=torch.uint8, device=dev)
    cap = cfg["rank_cap"]
    out = (torch.empty((cap, cfg["m"]), dtype=torch.complex128, device=dev),
           torch.empty(cap, dtype=torch.float64, device=dev),
           torch.empty((cap, cfg["n"]), dtype=torch.complex128, device=dev))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        res = B.compress(ctx, spec, opts, ws=ws, out=out)
    torch.cuda.synchronize(dev)
    # accounting from the (deterministic) pivot records of the last run
    L = cfg["levels"]
    traces, sizes = _leaf_records(B, spec, opts, ws, cfg["m"], cfg["n"], L)
    entries, flops = leaf_accounting(traces, sizes, cfg["d"], True)
    rank = res.rank

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    step_ms, baca_ms, recomp_ms, merge_ms = [], [], [], []
    launches = 0
    with ClockSampler(dev.index) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = B.compress(ctx, spec, opts, ws=ws, out=out)
            e1.record(stream)
            (tb, tr, tm, tt), launches = B.phase_times(ctx)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            baca_ms.append(tb)
            recomp_ms.append(tr)
            merge_ms.append(tm)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    ms_max = max_over_ranks(float(np.mean(step_ms)), world, dev)
    value = job_throughput(entries, ms_max / 1e3, world)

    # end to end through the C ABI with host buffers: pinned inputs -> device,
    # compress, factors -> pinned host, every step
    xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    yh = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
    xd = torch.empty_like(xh, device=dev)
    yd = torch.empty_like(yh, device=dev)
    spec_e2e = B.helmholtz(xd, yd, cfg["k"])
    Uh = torch.empty((cap, cfg["m"]), dtype=torch.complex128).pin_memory()
    Sh = torch.empty(cap, dtype=torch.float64).pin_memory()
    Vh = torch.empty((cap, cfg["n"]), dtype=torch.complex128).pin_memory()
    opts_e2e = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=cfg["seed"], rank_cap=cap,
                       leaf_rank_cap=cfg["leaf_rank_cap"])
    e2e_steps = max(1, min(args.steps, 5))
    B.compress(ctx, spec_e2e, opts_e2e, ws=ws, out=out)  # untimed: the binding's one-time argument checks
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(e2e_steps):
        xd.copy_(xh, non_blocking=True)
        yd.copy_(yh, non_blocking=True)
        r = B.compress(ctx, spec_e2e, opts_e2e, ws=ws, out=out)
        k = r.rank
        Uh[:k].copy_(out[0][:k], non_blocking=True)
        Sh[:k].copy_(out[1][:k], non_blocking=True)
        Vh[:k].copy_(out[2][:k], non_blocking=True)
        torch.cuda.synchronize(dev)
        h2d = xh.numel() * 8 + yh.numel() * 8
        d2h = k * (cfg["m"] + cfg["n"]) * 16 + k * 8
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    e2e_value = job_throughput(entries, e2e_s, world)

    # per-kernel device times of one more profiled compression (CUDA events
    # around every launch on the call's stream) and the rooflines
    phases = {"leaf_baca_ms": float(np.mean(baca_ms)), "leaf_recompression_ms": float(np.mean(recomp_ms)),
              "merge_ms": float(np.mean(merge_ms))}
    res = B.compress(ctx, spec, opts, ws=ws, out=out)
    torch.cuda.synchronize(dev)
    ktimes = B.kernel_times(ctx)
    stage_ms = {}
    for kname, st, _, kms in B.launch_times(ctx):
        key = "leaf_baca" if st < 0 else "stage%d" % st
        stage_ms.setdefault(key, {}).setdefault(kname, 0.0)
        stage_ms[key][kname] += kms
    plan = B.plan_json(spec, opts)
    dims = task_dims(ws, plan)
    jac_own = jacobi_accounting(ws, plan, True)
    jac_8d = jacobi_flops_8d(dims, True)
    whole_8d = whole_flops_8d(traces, sizes, cfg["d"], dims, True)
    jac_stages = jacobi_stage_stats(ws, plan)
    probe = B.fp64_probe()
    peak_note = ("FP64 peak derived from 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz; live probe DFMA %.3f, "
                 "DMMA %.3f TFLOP/s" % probe)
    dominant = max(ktimes, key=lambda kk: ktimes[kk][0])
    traffic = TRAFFIC_PER_LAUNCH.get(args.workload, {})
    qr_fl, qa_fl = dense_flops(dims, True)
    work = {"baca_leaf_kernel": flops, "jacobi_kernel": jac_8d, "qr_kernel": qr_fl, "qapply_kernel": qa_fl}
    roofs = {kn: roofline_of(kn, fl, ktimes, traffic.get(kn), peak_note) for kn, fl in work.items()}
    counts = {"jacobi_kernel": "20 r^3 per leaf core, 20 (2s)^3 per merge core, x4 complex",
              "qr_kernel": "2 m k^2 - 2 k^3 / 3 per Householder QR of m x k (geqrf count), x4 complex",
              "qapply_kernel": ("4 m k s - 2 k^2 s per application of k reflectors of m rows to s columns "
                                "(ormqr count), x4 complex; its event time overlaps the block products "
                                "running beside it on the auxiliary stream"),
              "baca_leaf_kernel": "the leaf BACA's own count from the pivot tape"}
    for kn in roofs:
        roofs[kn]["flop_count"] = counts[kn]
    roof = dict(roofs.get(dominant, roofs["jacobi_kernel"]), dominant_kernel=dominant)
    if roof["kernel"] == "jacobi_kernel":
        own = roofline_of("jacobi_kernel", jac_own, ktimes)
        roof["frac_by_kernel_sweeps"] = own["frac"]
    roof["frac_by_kernel"] = {kn: rr["frac"] for kn, rr in roofs.items()}
    whole = {"flops": whole_8d, "ms": ms_max, "achieved": whole_8d / (ms_max / 1e3) / 1e12,
             "frac": whole_8d / (ms_max / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "peak": FP64_PEAK_TFLOPS,
             "unit": "TFLOP/s", "flop_count": "leaf and merge work count of the measurement plan (r, s measured)"}
    return dict(value=value, ms=ms_max, entries=entries, flops=flops, rank=rank, phases=phases, roof=roof,
                roof_baca=roofs["baca_leaf_kernel"], kernel_ms={kk: v[0] for kk, v in ktimes.items()},
                jacobi_stages=jac_stages, whole=whole, stage_ms=stage_ms,
                launches=launches, clocks=clk.summary(), wall=wall, e2e=dict(value=e2e_value, unit="entries/s",
                h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, seconds_per_step=e2e_s), x=x, y=y)


# ------------------------------------------------------------------ the other workloads
def bench_cfg1(args, dev, flush, stream):
    """Gaussian 2000^2, d = 8, 4 x 4 leaves, eps = 1e-6."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs
    x, y = inputs.gaussian_pair(seed=0, m=2000, n=2000)
    ctx = B.Context()
    spec = B.gaussian(x, y, 1.0)
    opts = mk_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256)
    r = measure_single(B, ctx, spec, opts, 128, 2000, 2000, 2, 8, False, max(3, min(args.steps, 10)),
                       max(3, args.warmup), flush, stream, dev)
    err = B.rel_error(ctx, spec, r["res"])
    torch.cuda.synchronize(dev)
    whole = r["whole_flops"] / (r["ms"] / 1e3) / 1e12
    # the same call captured into a CUDA graph on its first run and replayed
    # (no host planning or synchronisation between stages)
    gopts = mk_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256, flags=B.FLAG_GRAPH)
    gws = torch.empty(B.workspace_size(spec.gen, gopts), dtype=torch.uint8, device=dev)
    gout = (torch.empty((128, 2000), dtype=torch.float64, device=dev), torch.empty(128, dtype=torch.float64, device=dev),
            torch.empty((128, 2000), dtype=torch.float64, device=dev))
    gms, gres = _timed_calls(lambda: B.compress(ctx, spec, gopts, ws=gws, out=gout), max(3, min(args.steps, 10)),
                             max(3, args.warmup), flush, stream)
    assert gres.rank == r["rank"]
    # the Frobenius truncation rule (HBACA_FLAG_FROB): budget eps / sqrt(2L + 1)
    # per truncation instead of the eps-rank
    fopts = mk_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256, flags=B.FLAG_FROB)
    fws = torch.empty(B.workspace_size(spec.gen, fopts), dtype=torch.uint8, device=dev)
    fout = (torch.empty((128, 2000), dtype=torch.float64, device=dev), torch.empty(128, dtype=torch.float64, device=dev),
            torch.empty((128, 2000), dtype=torch.float64, device=dev))
    fms, fres = _timed_calls(lambda: B.compress(ctx, spec, fopts, ws=fws, out=fout), max(3, min(args.steps, 10)),
                             max(3, args.warmup), flush, stream)
    ferr = B.rel_error(ctx, spec, fres)
    torch.cuda.synchronize(dev)
    return {"workload": "gaussian_f64_2000_d8_L2_eps1e-6", "ms": r["ms"], "ms_graph_replay": gms,
            "frob_truncation": {"ms": fms, "rank": fres.rank, "rel_error": ferr},
            "entries_per_s": r["entries"] / (r["ms"] / 1e3),
            "rank": r["rank"], "rel_error": err,
            "roofline_whole": {"achieved": whole, "frac": whole / FP64_PEAK_TFLOPS, "flops": r["whole_flops"],
                               "frac_graph_replay": r["whole_flops"] / (gms / 1e3) / 1e12 / FP64_PEAK_TFLOPS},
            "roofline_leaf_baca": roofline_of("baca_leaf_kernel", r["leaf_flops"], r["ktimes"]),
            "phases_ms": r["phases"], "gpu_launches": r["launches"],
            "kernel_ms": {kk: v[0] for kk, v in r["ktimes"].items()}}


def bench_cfg2_kd(args, dev, flush, stream):
    """The benchmark matrix with both point sets in KD-tree order (the
    setting of the paper's experiments, Sec. 5): the same matrix up to a
    permutation of rows and columns, whose leaves are spatial cells."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs
    cfg = WORKLOADS["helmholtz20000"]
    x, y = inputs.sphere_pair(seed=cfg["seed"], m=cfg["m"], n=cfg["n"])
    leaf = cfg["m"] >> cfg["levels"]
    xo, yo = x[B.kdtree_order(x, leaf)], y[B.kdtree_order(y, leaf)]
    ctx = B.Context()
    spec = B.helmholtz(xo, yo, cfg["k"])
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=cfg["seed"], rank_cap=cfg["rank_cap"],
                   leaf_rank_cap=cfg["leaf_rank_cap"])
    r = measure_single(B, ctx, spec, opts, cfg["rank_cap"], cfg["m"], cfg["n"], cfg["levels"], cfg["d"], True,
                       max(3, min(args.steps, 5)), 3, flush, stream, dev)
    err = B.rel_error(ctx, spec, r["res"])
    torch.cuda.synchronize(dev)
    return {"workload": cfg["workload"] + "_kdtree_order", "ms": r["ms"], "entries_per_s": r["entries"] / (r["ms"] / 1e3),
            "rank": r["rank"], "rel_error": err, "leaf_rank_max": r["res"].res.leaf_rank_max,
            "phases_ms": r["phases"], "kernel_ms": {kk: v[0] for kk, v in r["ktimes"].items()}}


def bench_cfg3(args, dev, flush, stream):
    """Coherent sparse product 50000^2 (K = 50, 1% density, rank-5 dense
    term), d = 32, 32 x 32 leaves, eps = 1e-8; plain ACA (d = 1) beside it."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs
    sp = inputs.sparse_product(seed=2, m=50000, n=50000, K=50, density=0.01)
    ctx = B.Context()
    spec = B.sparse_product(sp)
    out = {"workload": "sparse_product_f64_50000_K50_d32_L5_eps1e-8"}
    for name, d in (("baca", 32), ("aca", 1)):
        opts = mk_opts(1e-8, d, 5, seed=2, rank_cap=1024, leaf_rank_cap=512)
        t0 = time.perf_counter()
        try:
            r = measure_single(B, ctx, spec, opts, 1024, 50000, 50000, 5, d, False, 3 if d > 1 else 2,
                               3 if d > 1 else 1, flush, stream, dev)
        except B.HbacaError as e:
            # the leaf stage ran; its records are in the workspace of a plain call
            ws = torch.empty(B.workspace_size(spec.gen, opts), dtype=torch.uint8, device=dev)
            try:
                B.compress(ctx, spec, opts, ws=ws)
            except B.HbacaError:
                pass
            tr0 = B.read_leaf_trace(spec, opts, ws, 0)
            out[name] = {"d": d, "error": str(e), "wall_s": time.perf_counter() - t0,
                         "leaf0_nu_over_mu": [t["nu"] / t["mu"] if t["mu"] > 0 else 0.0 for t in tr0["trace"]],
                         "leaf0_stop": tr0["stop"], "leaf0_rank": tr0["rank_baca"]}
            del ws
            torch.cuda.empty_cache()
            continue
        err = B.rel_error(ctx, spec, r["res"])
        torch.cuda.synchronize(dev)
        # convergence history of the first leaf (Sec. 5.1): nu_k / mu_k per
        # iteration, the estimate the stopping test nu < eps mu uses
        hist = [t["nu"] / t["mu"] if t["mu"] > 0 else 0.0 for t in r["traces"][0]["trace"]]
        out[name] = {"d": d, "ms": r["ms"], "rank": r["rank"], "rel_error": err, "wall_s": time.perf_counter() - t0,
                     "leaf0_nu_over_mu": hist, "leaf0_stop": r["traces"][0]["stop"],
                     "entries_per_s": r["entries"] / (r["ms"] / 1e3), "leaf_rank_max": r["res"].res.leaf_rank_max,
                     "leaf_iters_max": r["res"].res.leaf_iters_max,
                     "kernel_ms": {kk: v[0] for kk, v in r["ktimes"].items()}, "phases_ms": r["phases"]}
        if d > 1:
            whole = r["whole_flops"] / (r["ms"] / 1e3) / 1e12
            out[name]["roofline_whole"] = {"achieved": whole, "frac": whole / FP64_PEAK_TFLOPS}
        del r
        torch.cuda.empty_cache()
    return out


def batched_measure(nblocks, loop_blocks, steps, warmup, flush, stream, dev):
    """hbaca_compress_batched over `nblocks` Gaussian blocks (autotuned leaf
    cluster, CUDA-graph replay) against the plain loop of one hbaca_compress
    per block, timed on the first `loop_blocks` blocks and scaled by the block
    count."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs
    cfg = WORKLOADS["batched4096"]
    blocks = inputs.batched_blocks(seed=cfg["seed"], nblocks=nblocks)
    ctx = B.Context()
    specs = [B.gaussian(x, y, h) for (x, y, h) in blocks]
    entries = float(sum(x.shape[0] * y.shape[0] for (x, y, _) in blocks))
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                   leaf_rank_cap=cfg["leaf_rank_cap"])
    batch = B.Batch(ctx, specs, opts)
    tuned_cluster, tuned_ms = batch.autotune()
    batch.opts.flags = B.FLAG_GRAPH | EXTRA_FLAGS
    ms, _ = _timed_calls(batch.run, steps, max(warmup, 1), flush, stream)
    ranks = batch.ranks()
    # phase split and launch count from one profiled (uncaptured) call
    pctx = B.Context()
    pb = B.Batch(pctx, specs, mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                                      leaf_rank_cap=cfg["leaf_rank_cap"], flags=B.FLAG_PROFILE,
                                      cluster=tuned_cluster), ws=batch.ws)
    pb.run()
    (tb, tr, tm, tt), launches = B.phase_times(pctx)
    ws_gib = batch.ws.numel() / 2 ** 30
    del pb, batch
    torch.cuda.empty_cache()
    lspecs = specs[:max(0, min(loop_blocks, nblocks))]
    lms = float("nan")
    loop_ranks = []
    if lspecs:
        lopts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                        leaf_rank_cap=cfg["leaf_rank_cap"])
        lws = torch.empty(max(B.workspace_size(s.gen, lopts) for s in lspecs), dtype=torch.uint8, device=dev)
        mmax, nmax, cap = max(s.m for s in lspecs), max(s.n for s in lspecs), cfg["rank_cap"]
        lout = (torch.empty(cap * mmax, dtype=torch.float64, device=dev),
                torch.empty(cap, dtype=torch.float64, device=dev),
                torch.empty(cap * nmax, dtype=torch.float64, device=dev))

        def loop():
            rk = []
            for s in lspecs:
                c = min(cap, s.m, s.n)
                o = (lout[0][:c * s.m].view(c, s.m), lout[1][:c], lout[2][:c * s.n].view(c, s.n))
                rk.append(B.compress(ctx, s, lopts, ws=lws, out=o).rank)
            return rk
        lms, loop_ranks = _timed_calls(loop, 1, 1, flush, stream)
        lms *= nblocks / len(lspecs)
    return {"workload": cfg["workload"].replace("4096", str(nblocks)), "batched_ms": ms,
            "per_block_loop_ms": lms, "speedup": lms / ms,
            "loop_timing": "%d of %d blocks timed, scaled by the block count" % (len(lspecs), nblocks),
            "entries_per_s": entries / (ms / 1e3), "batched_form": "one call, replayed CUDA graph",
            "autotuned_leaf_cluster": tuned_cluster, "autotune_baca_ms": tuned_ms,
            "phases_ms": {"leaf_baca_ms": tb, "leaf_recompression_ms": tr, "merge_ms": tm},
            "gpu_launches": launches, "ranks": {"max": max(ranks), "mean": float(np.mean(ranks)),
                                                "loop_mean": float(np.mean(loop_ranks)) if loop_ranks else None},
            "workspace_gib": ws_gib}


def grad_measure(steps, warmup, flush, stream, dev):
    """Differentiated workload: forward = taped compression + y = U(S(VX)),
    backward = dL/dh, dL/dx, dL/dy, dL/dX of L = 0.5 ||y||^2."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs
    cfg = WORKLOADS["grad16384"]
    x, y = inputs.gaussian_pair(seed=cfg["seed"], m=cfg["m"], n=cfg["n"])
    X = torch.from_numpy(inputs.rhs(cfg["seed"] + 1, cfg["n"], cfg["nrhs"])).to(dev)
    ctx = B.Context()
    spec = B.gaussian(x, y, cfg["h"])
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=cfg["seed"], rank_cap=cfg["rank_cap"],
                   leaf_rank_cap=cfg["leaf_rank_cap"], flags=B.FLAG_TAPE)
    plain = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=cfg["seed"], rank_cap=cfg["rank_cap"],
                    leaf_rank_cap=cfg["leaf_rank_cap"])
    ws = torch.empty(B.workspace_size(spec.gen, opts), dtype=torch.uint8, device=dev)
    wsp = torch.empty(B.workspace_size(spec.gen, plain), dtype=torch.uint8, device=dev)

    def timed(fn):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), o

    fwd, bwd, fwd_plain = [], [], []
    comp = grads = None
    for it in range(warmup + steps):
        tf, (comp, Y) = timed(lambda: (lambda c: (c, B.apply(ctx, spec, c, X)))(B.compress(ctx, spec, opts, ws=ws)))
        tb, grads = timed(lambda: B.apply_backward(ctx, spec, opts, comp, X, Y))
        tp, _ = timed(lambda: B.compress(ctx, spec, plain, ws=wsp))
        if it >= warmup:
            fwd.append(tf)
            bwd.append(tb)
            fwd_plain.append(tp)
    f, b = float(np.mean(fwd)), float(np.mean(bwd))
    return {"workload": cfg["workload"], "forward_ms": f, "backward_ms": b, "bwd_over_fwd": b / f,
            "forward_untaped_compress_ms": float(np.mean(fwd_plain)), "rank": comp.rank, "dL_dh": float(grads[0])}


def extra_configs(args, dev):
    """The other workloads' compact keys; a failure is recorded, not raised."""
    import torch
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    jobs = [("cfg1", lambda: bench_cfg1(args, dev, flush, stream)),
            ("cfg2_kd_order", lambda: bench_cfg2_kd(args, dev, flush, stream)),
            ("cfg3", lambda: bench_cfg3(args, dev, flush, stream)),
            ("cfg4", lambda: batched_measure(4096, args.loop_blocks, 2, 1, flush, stream, dev)),
            ("cfg5", lambda: grad_measure(3, 2, flush, stream, dev))]
    for name, fn in jobs:
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # noqa: BLE001 - recorded in the line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
    return out


def run_grad(args):
    """One step = forward (taped compression + apply) and backward of the
    differentiated workload; reports both times and their ratio."""
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(dev.index) as clk:
        r = grad_measure(args.steps, args.warmup, flush, torch.cuda.current_stream(dev), dev)
    cfg = WORKLOAD
    line = {"metric": METRIC, "value": r["bwd_over_fwd"], "unit": "backward ms / forward ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["forward_ms"] + r["backward_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="flushed between timed calls (512 MiB write)", parallelism="1 GPU"),
            "clocks": clk.summary()}
    line.update({k: v for k, v in r.items() if k != "workload"})
    print(json.dumps(line))


def run_gradbatch(args):
    """One step = batched taped compression + apply per block (forward) and one
    batched reverse pass (backward); reports both times and their ratio."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs

    cfg = WORKLOAD
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    blocks = inputs.grad_blocks(seed=cfg["seed"], nblocks=cfg["nblocks"], h=cfg["h"])
    ctx = B.Context()
    specs = [B.gaussian(x, y, h) for (x, y, h) in blocks]
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                   leaf_rank_cap=cfg["leaf_rank_cap"], flags=B.FLAG_TAPE)
    bt = B.Batch(ctx, specs, opts)
    Xs = [torch.from_numpy(inputs.rhs(cfg["seed"] + 1 + b, s.n, cfg["nrhs"])).to(dev) for b, s in enumerate(specs)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    def forward():
        bt.run()
        return [B.apply(ctx, s, c, X) for s, c, X in zip(specs, bt.results(), Xs)]

    fwd, bwd = [], []
    with ClockSampler(dev.index) as clk:
        for it in range(args.warmup + args.steps):
            tf, Ys = timed(forward)
            tb, _ = timed(lambda: B.apply_backward_batched(bt, Xs, Ys, want_dX=True))
            if it >= args.warmup:
                fwd.append(tf)
                bwd.append(tb)
    f, b = float(np.mean(fwd)), float(np.mean(bwd))
    ranks = bt.ranks()
    line = {"metric": METRIC, "value": b / f, "unit": "backward ms / forward ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f + b, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="flushed between timed calls (512 MiB write)", parallelism="1 GPU"),
            "forward_ms": f, "backward_ms": b, "ranks": {"max": max(ranks), "mean": float(np.mean(ranks))},
            "clocks": clk.summary()}
    print(json.dumps(line))


def run_batched(args):
    """One step = hbaca_compress_batched over all blocks; the plain per-block
    loop (one hbaca_compress per block, same d, eps, leaf size and caps) is
    timed beside it on the same stream."""
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    nblocks = args.nblocks or WORKLOAD["nblocks"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(dev.index) as clk:
        r = batched_measure(nblocks, 0 if args.no_loop else min(args.loop_blocks, nblocks), args.steps,
                            args.warmup, flush, torch.cuda.current_stream(dev), dev)
    cfg = dict(WORKLOAD, nblocks=nblocks)
    line = {"metric": METRIC, "value": r["entries_per_s"], "unit": "matrix entries compressed/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["batched_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="flushed between timed steps (512 MiB write)", parallelism="1 GPU"),
            "batched_vs_loop": r, "clocks": clk.summary()}
    print(json.dumps(line))


def run_reference(args, rank):
    """The oracle arm: each step is the oracle H-BACA (all leaves and merges,
    spawned processes of one BLAS thread) of the leading 4 x 4 leaves of the
    benchmark matrix (rows and columns 0..4999: the same leaves, leaf sizes
    and initial column blocks as the full workload, two merge levels)."""
    if rank != 0:
        return
    from paper_1901_06101_gb300 import inputs
    cfg = WORKLOAD
    x, y = inputs.sphere_pair(seed=cfg["seed"], m=cfg["m"], n=cfg["n"])
    L = cfg["levels"]
    Ls = min(2, L)
    ms_, ns_ = sum(s for _, s in leaf_spans(cfg["m"], L)[:1 << Ls]), sum(s for _, s in leaf_spans(cfg["n"], L)[:1 << Ls])
    op = OraclePool()
    vals, secs = [], []
    try:
        for i in range(args.warmup + args.steps):
            entries, dt, _ = oracle_hbaca_pool(op, x[:ms_], y[:ns_], cfg["k"], Ls, cfg["d"], cfg["eps"], cfg["seed"])
            if i >= args.warmup:
                vals.append(entries / dt)
                secs.append(dt)
    finally:
        op.close()
    value = float(np.mean(vals))
    desc = ("oracle H-BACA (all %d leaves, every merge level; Alg. 2, Sec. 3.2, Alg. 3) of the leading %dx%d block "
            "of the workload matrix (the workload's own %dx%d leaves), %d spawned processes x 1 BLAS thread"
            % (4 ** Ls, ms_, ns_, ms_ >> Ls, ns_ >> Ls, op.procs))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": dict({k: v for k, v in cfg.items() if k != "k"}, k="4*pi", l2="n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": op.procs, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    global WORKLOAD, EXTRA_FLAGS
    args = parse()
    WORKLOAD = WORKLOADS[args.workload]
    if args.single_cluster:
        EXTRA_FLAGS = 16  # HBACA_FLAG_SINGLE_CLUSTER
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    single = {"grad16384": run_grad, "gradbatch256": run_gradbatch, "batched4096": run_batched}
    if args.workload in single:
        if args.impl == "reference" or world > 1:
            raise SystemExit("this workload is a single-GPU comparison of two forms of the same GPU path")
        single[args.workload](args)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(r["x"], r["y"], WORKLOAD)
    extra = {}
    if world == 1 and not args.no_extra and args.workload == "helmholtz20000":
        import torch
        extra = extra_configs(args, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
    cfg = dict({k: v for k, v in WORKLOAD.items() if k != "k"}, k="4*pi",
               l2="flushed between timed steps (512 MiB write)", parallelism="replicas" if world > 1 else "1 GPU")
    line = {"metric": METRIC, "value": r["value"], "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": cfg,
            "roofline": r["roof"], "roofline_whole": r["whole"], "cpu_baseline": cpu, "e2e": r["e2e"],
            "gpu_launches": r["launches"], "clocks": r["clocks"], "phases_ms": r["phases"], "rank": r["rank"],
            "roofline_leaf_baca": r["roof_baca"], "kernel_ms": r["kernel_ms"],
            "jacobi_stages": r["jacobi_stages"], "stage_kernel_ms": r["stage_ms"], "entries_per_step": r["entries"]}
    line.update(extra)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
