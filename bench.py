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
TRAFFIC_PER_LAUNCH = {"helmholtz20000": {"jacobi_kernel": 13.78e6}}


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
    every sweep forms the three inner products of each of the nc (nc - 1) / 2
    column pairs over the mr rows of the core, and every applied rotation
    updates both columns of the core (mr rows), and of the accumulated
    rotation (nc rows) when the call is taped (``accumulates``).  Per element:
    inner products 16 flops (complex) / 6 (real), rotation 18 / 7."""
    import torch
    fd, fr = (16.0, 18.0) if complex_ else (6.0, 7.0)
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
            total += nsw * nc * (nc - 1) / 2 * mr * fd + float(rot) * (mr + (nc if accumulates else 0)) * fr
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
def _oracle_leaf(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    x, y, k, r0, mr, c0, nc, d, eps, seed, a, b = args
    from oracle import baca as ob
    from oracle import generators as og
    from oracle import sampler as osamp
    g = og.Window(og.Helmholtz(x, y, k), r0, mr, c0, nc)
    res = ob.baca(g, d, eps, seed=seed, bid=osamp.block_id(0, a, b))
    ob.recompress(res["U"], res["V"], eps)
    return sum(mr * len(t["J"]) + len(t["I"]) * nc for t in res["trace"])


def _warm(_):
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle.baca  # noqa: F401
    return 0


def oracle_sample(x, y, cfg, seconds, max_procs=None):
    """The CPU oracle (leaf BACA + re-compression of Alg. 2 / Sec. 3.2) on a
    bounded sample of the workload's leaves, processes spawned, one BLAS thread
    each.  Returns (entries/s, cores used, description)."""
    import multiprocessing as mp
    L = cfg["levels"]
    rows = leaf_spans(cfg["m"], L)
    cols = leaf_spans(cfg["n"], L)
    nb = 1 << L
    cores = len(os.sched_getaffinity(0))
    procs = max(1, min(cores, max_procs or cores))
    ctx = mp.get_context("spawn")
    jobs = []
    order = np.random.default_rng(0).permutation(nb * nb)
    for leaf in order:
        a, b = divmod(int(leaf), nb)
        jobs.append((x, y, cfg["k"], rows[a][0], rows[a][1], cols[b][0], cols[b][1], cfg["d"], cfg["eps"],
                     cfg["seed"], a, b))
    done = 0
    entries = 0
    with ctx.Pool(procs) as pool:
        pool.map(_warm, range(procs))  # interpreter start-up outside the timed sample
        t0 = time.perf_counter()
        while done < len(jobs) and time.perf_counter() - t0 < seconds:
            batch = jobs[done:done + procs]
            entries += sum(pool.map(_oracle_leaf, batch))
            done += len(batch)
    dt = time.perf_counter() - t0
    desc = ("oracle leaf BACA + SVD re-compression (Alg. 2, Sec. 3.2) on %d of %d leaves (%dx%d each), "
            "%d spawned processes x 1 BLAS thread; merges not sampled" % (done, nb * nb, rows[0][1], cols[0][1], procs))
    return entries / dt, procs, desc, dt


# ------------------------------------------------------------------ GPU arm
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
    nb = 1 << L
    rows = leaf_spans(cfg["m"], L)
    cols = leaf_spans(cfg["n"], L)
    traces, sizes = [], []
    for leaf in range(nb * nb):
        traces.append(B.read_leaf_trace(spec, opts, ws, leaf))
        a, b = divmod(leaf, nb)
        sizes.append((rows[a][1], cols[b][1]))
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

    # per-kernel device times of the last timed compression (CUDA events around
    # every launch on the call's stream) and the roofline of the dominant one
    phases = {"leaf_baca_ms": float(np.mean(baca_ms)), "leaf_recompression_ms": float(np.mean(recomp_ms)),
              "merge_ms": float(np.mean(merge_ms))}
    res = B.compress(ctx, spec, opts, ws=ws, out=out)
    torch.cuda.synchronize(dev)
    ktimes = B.kernel_times(ctx)
    plan = B.plan_json(spec, opts)
    jac_flops = jacobi_accounting(ws, plan, True)
    jac_stages = jacobi_stage_stats(ws, plan)
    probe = B.fp64_probe()
    peak_note = ("FP64 peak derived from 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz; live probe DFMA %.3f, "
                 "DMMA %.3f TFLOP/s" % probe)
    dominant = max(ktimes, key=lambda k: ktimes[k][0])
    work = {"baca_leaf_kernel": flops, "jacobi_kernel": jac_flops}
    roofs = {}
    for kname, fl in work.items():
        kms, kl = ktimes[kname]
        ach = fl / (kms / 1e3) / 1e12
        traffic = TRAFFIC_PER_LAUNCH.get(args.workload, {}).get(kname)
        roofs[kname] = {"bound": "alu", "kernel": kname, "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic, "flops_per_launch": fl / max(kl, 1),
                        "ms_per_launch": kms / max(kl, 1), "launches": kl, "peak_note": peak_note}
    roof = roofs.get(dominant, roofs["jacobi_kernel"])
    roof = dict(roof, dominant_kernel=dominant)
    return dict(value=value, ms=ms_max, entries=entries, flops=flops, rank=rank, phases=phases, roof=roof,
                roof_baca=roofs["baca_leaf_kernel"], kernel_ms={k: v[0] for k, v in ktimes.items()},
                jacobi_stages=jac_stages,
                launches=launches, clocks=clk.summary(), wall=wall, e2e=dict(value=e2e_value, unit="entries/s",
                h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, seconds_per_step=e2e_s), x=x, y=y)


def run_grad(args):
    """One step = forward (taped compression + apply) and backward of the
    differentiated workload; reports both times and their ratio."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs

    cfg = WORKLOAD
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
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

    fwd, bwd, fwd_plain = [], [], []
    comp = Y = None
    with ClockSampler(dev.index) as clk:
        for it in range(args.warmup + args.steps):
            tf, (comp, Y) = timed(lambda: (lambda c: (c, B.apply(ctx, spec, c, X)))(B.compress(ctx, spec, opts, ws=ws)))
            tb, grads = timed(lambda: B.apply_backward(ctx, spec, opts, comp, X, Y))
            tp, _ = timed(lambda: B.compress(ctx, spec, plain, ws=wsp))
            if it >= args.warmup:
                fwd.append(tf)
                bwd.append(tb)
                fwd_plain.append(tp)
    f, b = float(np.mean(fwd)), float(np.mean(bwd))
    dh = float(grads[0])
    line = {"metric": METRIC, "value": b / f, "unit": "backward ms / forward ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f + b, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="flushed between timed calls (512 MiB write)", parallelism="1 GPU"),
            "forward_ms": f, "backward_ms": b, "forward_untaped_compress_ms": float(np.mean(fwd_plain)),
            "rank": comp.rank, "dL_dh": dh, "clocks": clk.summary()}
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
    """One step = hbaca_compress_batched over all blocks.  The plain per-block
    loop (one hbaca_compress per block, same d, eps, leaf size and caps) is
    timed beside it on the same stream."""
    import torch
    from paper_1901_06101_gb300 import binding as B
    from paper_1901_06101_gb300 import inputs

    cfg = WORKLOAD
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if args.nblocks:
        cfg = dict(cfg, nblocks=args.nblocks, workload=cfg["workload"].replace("4096", str(args.nblocks)))
    blocks = inputs.batched_blocks(seed=cfg["seed"], nblocks=cfg["nblocks"])
    ctx = B.Context()
    specs = [B.gaussian(x, y, h) for (x, y, h) in blocks]
    entries = float(sum(x.shape[0] * y.shape[0] for (x, y, _) in blocks))
    # the batched arm: leaf cluster size from the autotuner, the call captured
    # into a CUDA graph on its first (warm-up) run and replayed afterwards
    opts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                       leaf_rank_cap=cfg["leaf_rank_cap"])
    batch = B.Batch(ctx, specs, opts)
    tuned_cluster, tuned_ms = batch.autotune()
    batch.opts.flags = B.FLAG_GRAPH | EXTRA_FLAGS
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        batch.run()
    torch.cuda.synchronize(dev)
    ranks = batch.ranks()
    step_ms, phase = [], []
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.run()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    ms = float(np.mean(step_ms))
    # phase split and launch count from one profiled (uncaptured) call
    pctx = B.Context()
    pb = B.Batch(pctx, specs, mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                                          leaf_rank_cap=cfg["leaf_rank_cap"], flags=B.FLAG_PROFILE,
                                          cluster=tuned_cluster), ws=batch.ws)
    pb.run()
    (tb, tr, tm, tt), launches = B.phase_times(pctx)
    # the plain loop: one compress per block, shared workspace and outputs
    lopts = mk_opts(cfg["eps"], cfg["d"], cfg["levels"], seed=0, rank_cap=cfg["rank_cap"],
                        leaf_rank_cap=cfg["leaf_rank_cap"])
    wsz = max(B.workspace_size(s.gen, lopts) for s in specs)
    lws = torch.empty(wsz, dtype=torch.uint8, device=dev)
    mmax = max(s.m for s in specs)
    nmax = max(s.n for s in specs)
    cap = cfg["rank_cap"]
    lout = (torch.empty(cap * mmax, dtype=torch.float64, device=dev),
            torch.empty(cap, dtype=torch.float64, device=dev),
            torch.empty(cap * nmax, dtype=torch.float64, device=dev))

    def loop():
        rk = []
        for s in specs:
            c = min(cap, s.m, s.n)
            out = (lout[0][:c * s.m].view(c, s.m), lout[1][:c], lout[2][:c * s.n].view(c, s.n))
            rk.append(B.compress(ctx, s, lopts, ws=lws, out=out).rank)
        return rk

    loop_ranks = loop() if not args.no_loop else [0]  # warm-up
    loop_steps = max(1, min(args.steps, 2)) if not args.no_loop else 0
    loop_ms = [float("nan")]
    for _ in range(loop_steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop()
        e1.record(stream)
        e1.synchronize()
        loop_ms.append(e0.elapsed_time(e1))
    lms = float(np.mean(loop_ms[1:] if loop_steps else loop_ms))
    line = {"metric": METRIC, "value": entries / (ms / 1e3), "unit": "matrix entries compressed/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="flushed between timed steps (512 MiB write)", parallelism="1 GPU"),
            "batched_vs_loop": {"batched_ms": ms, "per_block_loop_ms": lms, "speedup": lms / ms,
                                "loop_steps": loop_steps, "batched_form": "one call, replayed CUDA graph",
                                "autotuned_leaf_cluster": tuned_cluster, "autotune_baca_ms": tuned_ms},
            "phases_ms": {"leaf_baca_ms": tb, "leaf_recompression_ms": tr, "merge_ms": tm},
            "gpu_launches": launches, "clocks": clk.summary(),
            "ranks": {"max": max(ranks), "mean": float(np.mean(ranks)), "loop_mean": float(np.mean(loop_ranks))},
            "workspace_gib": batch.ws.numel() / 2 ** 30}
    print(json.dumps(line))


def main():
    global WORKLOAD, EXTRA_FLAGS
    args = parse()
    WORKLOAD = WORKLOADS[args.workload]
    if args.single_cluster:
        EXTRA_FLAGS = 16  # HBACA_FLAG_SINGLE_CLUSTER
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "grad16384":
        if args.impl == "reference" or world > 1:
            raise SystemExit("the gradient workload is a single-GPU forward/backward comparison")
        run_grad(args)
        return
    if args.workload == "gradbatch256":
        if args.impl == "reference" or world > 1:
            raise SystemExit("the gradient workload is a single-GPU forward/backward comparison")
        run_gradbatch(args)
        return
    if args.workload == "batched4096":
        if args.impl == "reference" or world > 1:
            raise SystemExit("the batched workload is a single-GPU comparison of the two call forms")
        run_batched(args)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        cfg = WORKLOAD
        from paper_1901_06101_gb300 import inputs
        x, y = inputs.sphere_pair(seed=cfg["seed"], m=cfg["m"], n=cfg["n"])
        per = max(5.0, min(60.0, 150.0 / max(1, args.steps + args.warmup)))
        vals = []
        for i in range(args.warmup + args.steps):
            v, cores, desc, dt = oracle_sample(x, y, cfg, per)
            if i >= args.warmup:
                vals.append(v)
        value = float(np.mean(vals))
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": dict({k: v for k, v in cfg.items() if k != "k"}, k="4*pi", l2="n/a (CPU)"),
                "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, cores, desc, dt = oracle_sample(r["x"], r["y"], WORKLOAD, args.cpu_seconds)
        cpu = {"value": v, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": dt}
    cfg = dict({k: v for k, v in WORKLOAD.items() if k != "k"}, k="4*pi",
               l2="flushed between timed steps (512 MiB write)", parallelism="replicas" if world > 1 else "1 GPU")
    line = {"metric": METRIC, "value": r["value"], "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": cfg,
            "roofline": r["roof"], "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["launches"],
            "clocks": r["clocks"], "phases_ms": r["phases"], "rank": r["rank"],
            "roofline_leaf_baca": r["roof_baca"], "kernel_ms": r["kernel_ms"],
            "jacobi_stages": r["jacobi_stages"], "entries_per_step": r["entries"]}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
