"""Thin Python binding of libhbaca.so (include/hbaca.h).

Argument marshalling only: every step of the compression runs in the CUDA
library.  PyTorch provides device memory and the stream.  There is no CPU
fallback: if the library is missing, ``lib()`` raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhbaca.so")

# hbaca_gen_kind
GEN_DENSE, GEN_GAUSSIAN, GEN_HELMHOLTZ, GEN_SPARSE_PRODUCT, GEN_LOWRANK, GEN_POLYNOMIAL, GEN_HANKEL2D = range(7)
# hbaca_dtype
F64, C128 = 0, 1
FLAG_ASYNC = 1
FLAG_PROFILE = 2
FLAG_TAPE = 4
FLAG_GRAPH = 8
FLAG_SINGLE_CLUSTER = 16
FLAG_FROB = 32
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "RANK_CAPACITY", 3: "CUDA", 4: "TIMEOUT",
          5: "NO_TAPE", 6: "NUMERICAL", 7: "WORKSPACE", 8: "NOT_CONVERGED"}
STOP = {0: "converged", 1: "iterations", 2: "no columns", 3: "no rows", 4: "capacity", 5: "numerical"}


class Gen(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("m", ctypes.c_int64), ("n", ctypes.c_int64),
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
        ("dim", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("h", ctypes.c_double), ("k", ctypes.c_double),
        ("a", ctypes.c_void_p), ("lda", ctypes.c_int64),
        ("lu", ctypes.c_void_p), ("lv", ctypes.c_void_p), ("lr", ctypes.c_int64),
        ("K", ctypes.c_int64),
        ("p_rowptr", ctypes.c_void_p), ("p_colidx", ctypes.c_void_p), ("p_val", ctypes.c_void_p),
        ("q_colptr", ctypes.c_void_p), ("q_rowidx", ctypes.c_void_p), ("q_val", ctypes.c_void_p),
        ("p2", ctypes.c_void_p), ("q2", ctypes.c_void_p),
        ("r2", ctypes.c_int32), ("pad1", ctypes.c_int32),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double), ("d", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("rank_cap", ctypes.c_int64), ("leaf_rank_cap", ctypes.c_int64),
        ("flags", ctypes.c_uint32), ("cluster", ctypes.c_int32), ("srrqr_f", ctypes.c_double),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64), ("S", ctypes.c_void_p),
        ("V", ctypes.c_void_p), ("ldv", ctypes.c_int64), ("d_rank", ctypes.c_void_p),
        ("rank", ctypes.c_int64), ("leaf_rank_max", ctypes.c_int32), ("leaf_iters_max", ctypes.c_int32),
    ]


class LeafTrace(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("rank_baca", ctypes.c_int32), ("rank", ctypes.c_int32),
        ("stop", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("d", ctypes.c_int32),
        ("I", ctypes.c_void_p), ("J", ctypes.c_void_p), ("jbar", ctypes.c_void_p),
        ("dI", ctypes.c_void_p), ("dJ", ctypes.c_void_p), ("dk", ctypes.c_void_p),
        ("nu", ctypes.c_void_p), ("mu", ctypes.c_void_p),
    ]


_LIB = None

# (name, restype, argtypes) for every function include/hbaca.h declares
SIGNATURES = [
    ("hbaca_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    ("hbaca_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("hbaca_workspace_size", ctypes.c_size_t, [ctypes.POINTER(Gen), ctypes.POINTER(Opts)]),
    ("hbaca_compress", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Gen), ctypes.POINTER(Opts),
                                      ctypes.POINTER(Result), ctypes.c_void_p, ctypes.c_void_p]),
    ("hbaca_read_leaf_trace", ctypes.c_int, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_void_p,
                                             ctypes.c_int64, ctypes.POINTER(LeafTrace), ctypes.c_void_p]),
    ("hbaca_debug_backward_json", ctypes.c_int64, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_void_p,
                                                   ctypes.c_int64, ctypes.c_char_p, ctypes.c_int64, ctypes.c_void_p]),
    ("hbaca_autotune_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Gen), ctypes.POINTER(Opts),
                                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    ("hbaca_kernel_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int32)]),
    ("hbaca_backward_workspace_size_batched", ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(Gen),
                                                                ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_int64,
                                                                ctypes.c_void_p]),
    ("hbaca_apply_backward_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Gen),
                                                    ctypes.POINTER(Opts), ctypes.POINTER(Result), ctypes.c_void_p,
                                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_size_t,
                                                    ctypes.c_void_p]),
    ("hbaca_apply_workspace_size", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    ("hbaca_apply", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Gen), ctypes.POINTER(Result), ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    ("hbaca_backward_workspace_size", ctypes.c_size_t, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_void_p,
                                                        ctypes.c_int64, ctypes.c_void_p]),
    ("hbaca_apply_backward", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Gen), ctypes.POINTER(Opts),
                                            ctypes.POINTER(Result), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("hbaca_compress_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Gen), ctypes.POINTER(Opts),
                                              ctypes.POINTER(Result), ctypes.c_void_p]),
    ("hbaca_workspace_size_batched", ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(Gen), ctypes.POINTER(Opts)]),
    ("hbaca_compress_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Gen),
                                              ctypes.POINTER(Opts), ctypes.POINTER(Result), ctypes.c_void_p,
                                              ctypes.c_void_p]),
    ("hbaca_read_leaf_trace_batched", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Gen), ctypes.POINTER(Opts),
                                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                                     ctypes.POINTER(LeafTrace), ctypes.c_void_p]),
    ("hbaca_debug_read_block", ctypes.c_int, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_void_p,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 4
     + [ctypes.c_void_p]),
    ("hbaca_debug_plan_json", ctypes.c_size_t, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_char_p,
                                                ctypes.c_size_t]),
    ("hbaca_phase_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32)]),
    ("hbaca_debug_set_jacobi_sweeps", ctypes.c_int32, [ctypes.c_int32]),
    ("hbaca_debug_set_jacobi_cluster", ctypes.c_int32, [ctypes.c_int32]),
    ("hbaca_debug_set_qr_cluster", ctypes.c_int32, [ctypes.c_int32]),
    ("hbaca_debug_set_jacobi_groups", ctypes.c_int32, [ctypes.c_int32]),
    ("hbaca_debug_set_qr_groups", ctypes.c_int32, [ctypes.c_int32]),
    ("hbaca_error_workspace_size", ctypes.c_size_t, [ctypes.c_int64]),
    ("hbaca_debug_launch_times", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_int32]),
    ("hbaca_kdtree_order", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_void_p]),
    ("hbaca_hmatrix_blocks", ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                              ctypes.c_int64]),
    ("hbaca_debug_read_leaf_factors", ctypes.c_int, [ctypes.POINTER(Gen), ctypes.POINTER(Opts), ctypes.c_void_p,
                                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
     + [ctypes.POINTER(ctypes.c_int64)] * 3 + [ctypes.c_void_p]),
    ("hbaca_debug_entries", ctypes.c_int, [ctypes.POINTER(Gen), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    ("hbaca_error_norms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Gen), ctypes.POINTER(Result), ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p]),
    ("hbaca_last_error", ctypes.c_char_p, []),
    ("hbaca_version", ctypes.c_char_p, []),
]


def lib():
    """Load libhbaca.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhbaca.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1901_06101_gb300.build); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class HbacaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hbaca status %s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


def check(code):
    if code != 0:
        raise HbacaError(code, lib().hbaca_last_error().decode())


class Context:
    """hbaca_ctx bound to the current CUDA device."""

    def __init__(self):
        self.ptr = ctypes.c_void_p()
        check(lib().hbaca_create(ctypes.byref(self.ptr)))

    def __del__(self):
        try:
            if self.ptr:
                lib().hbaca_destroy(self.ptr)
        except Exception:
            pass


def make_opts(eps, d, levels, seed=0, rank_cap=0, leaf_rank_cap=0, flags=0, cluster=0, srrqr_f=0.0):
    return Opts(eps=eps, d=d, levels=levels, seed=seed, rank_cap=rank_cap,
                leaf_rank_cap=leaf_rank_cap, flags=flags, cluster=cluster, srrqr_f=srrqr_f)


def workspace_size(gen, opts):
    n = lib().hbaca_workspace_size(ctypes.byref(gen), ctypes.byref(opts))
    if n == 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    return n


# ---------------------------------------------------------------- torch helpers
def _dev(t, dtype=None):
    import torch
    if dtype is not None:
        t = torch.as_tensor(t, dtype=dtype)
    t = torch.as_tensor(t)
    if not t.is_cuda:
        t = t.to("cuda")
    return t.contiguous()


class GenSpec:
    """A hbaca_gen plus the device tensors it points into (kept alive)."""

    def __init__(self, gen, keep):
        self.gen = gen
        self.keep = keep

    @property
    def m(self):
        return self.gen.m

    @property
    def n(self):
        return self.gen.n

    @property
    def complex(self):
        return self.gen.dtype == C128


def gaussian(x, y, h):
    import torch
    x = _dev(x, torch.float64)
    y = _dev(y, torch.float64)
    g = Gen(kind=GEN_GAUSSIAN, dtype=F64, m=x.shape[0], n=y.shape[0], x=x.data_ptr(), y=y.data_ptr(),
            dim=x.shape[1], h=float(h))
    return GenSpec(g, (x, y))


def helmholtz(x, y, k):
    import torch
    x = _dev(x, torch.float64)
    y = _dev(y, torch.float64)
    g = Gen(kind=GEN_HELMHOLTZ, dtype=C128, m=x.shape[0], n=y.shape[0], x=x.data_ptr(), y=y.data_ptr(),
            dim=x.shape[1], k=float(k))
    return GenSpec(g, (x, y))


def polynomial(x, y, h):
    """Polynomial kernel (x_i^t y_j + h)^2."""
    import torch
    x = _dev(x, torch.float64)
    y = _dev(y, torch.float64)
    g = Gen(kind=GEN_POLYNOMIAL, dtype=F64, m=x.shape[0], n=y.shape[0], x=x.data_ptr(), y=y.data_ptr(),
            dim=x.shape[1], h=float(h))
    return GenSpec(g, (x, y))


def hankel2d(x, y, k):
    """EFIE2D kernel H0^(2)(k ||x_i - y_j||) (complex128)."""
    import torch
    x = _dev(x, torch.float64)
    y = _dev(y, torch.float64)
    g = Gen(kind=GEN_HANKEL2D, dtype=C128, m=x.shape[0], n=y.shape[0], x=x.data_ptr(), y=y.data_ptr(),
            dim=x.shape[1], k=float(k))
    return GenSpec(g, (x, y))


def entries(spec, rows, cols):
    """hbaca_debug_entries: A(rows[t], cols[t]) from the device generators, as
    a numpy array."""
    import numpy as np
    import torch
    r = torch.as_tensor(np.asarray(rows, np.int64)).cuda()
    c = torch.as_tensor(np.asarray(cols, np.int64)).cuda()
    out = torch.empty(r.numel(), dtype=torch.complex128 if spec.complex else torch.float64, device="cuda")
    check(lib().hbaca_debug_entries(ctypes.byref(spec.gen), ctypes.c_void_p(r.data_ptr()),
                                    ctypes.c_void_p(c.data_ptr()), r.numel(), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out.cpu().numpy()


def dense(A):
    """A (m x n) numpy / torch array; stored column-major on the device."""
    import torch
    A = torch.as_tensor(A)
    cplx = A.is_complex()
    At = _dev(A.T.contiguous(), torch.complex128 if cplx else torch.float64)  # (n, m) row-major = A col-major
    g = Gen(kind=GEN_DENSE, dtype=C128 if cplx else F64, m=A.shape[0], n=A.shape[1], a=At.data_ptr(), lda=A.shape[0])
    return GenSpec(g, (At,))


def lowrank(LU, LV):
    import torch
    LU = torch.as_tensor(LU)
    LV = torch.as_tensor(LV)
    cplx = LU.is_complex() or LV.is_complex()
    dt = torch.complex128 if cplx else torch.float64
    LUt = _dev(LU.T.contiguous(), dt)  # column-major m x lr
    LVd = _dev(LV, dt)
    g = Gen(kind=GEN_LOWRANK, dtype=C128 if cplx else F64, m=LU.shape[0], n=LV.shape[1],
            lu=LUt.data_ptr(), lv=LVd.data_ptr(), lr=LU.shape[1])
    return GenSpec(g, (LUt, LVd))


def sparse_product(sp):
    """``sp``: paper_1901_06101_gb300.inputs.SparseProductInputs."""
    import torch
    t = [_dev(torch.as_tensor(a)) for a in (sp.p_rowptr, sp.p_colidx, sp.p_val, sp.q_colptr, sp.q_rowidx,
                                             sp.q_val, sp.P2, sp.Q2)]
    g = Gen(kind=GEN_SPARSE_PRODUCT, dtype=F64, m=sp.m, n=sp.n, K=sp.K,
            p_rowptr=t[0].data_ptr(), p_colidx=t[1].data_ptr(), p_val=t[2].data_ptr(),
            q_colptr=t[3].data_ptr(), q_rowidx=t[4].data_ptr(), q_val=t[5].data_ptr(),
            p2=t[6].data_ptr(), q2=t[7].data_ptr(), r2=sp.P2.shape[1])
    return GenSpec(g, tuple(t))


def _host_rank(res, opts):
    """The rank a synchronous call returned on the host.  HBACA_FLAG_ASYNC
    calls leave it at -1 (the rank goes to a device int); these helpers
    slice the factors by the rank, so they refuse that flag."""
    r = int(res.rank)
    if r < 0:
        raise HbacaError(1, "no host rank (HBACA_FLAG_ASYNC): these helpers need a synchronous call")
    return r


def error_norms(ctx, spec, comp, rows=None, stream=None):
    """hbaca_error_norms: (||A(I,:) - U(I,:) S V||_F^2, ||A(I,:)||_F^2) on the
    device over the rows I (all rows when None) of the compressed matrix
    ``comp`` (a Compressed from a synchronous call)."""
    import numpy as np
    import torch
    if rows is None:
        rp, nr = None, 0
    else:
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        rp, nr = rows.ctypes.data_as(ctypes.c_void_p), rows.size
    nbytes = lib().hbaca_error_workspace_size(nr)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * 2)()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib().hbaca_error_norms(ctx.ptr, ctypes.byref(spec.gen), ctypes.byref(comp.res), rp, nr, out,
                                  ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.c_void_p(stream)))
    return out[0], out[1]


def rel_error(ctx, spec, comp, rows=None):
    """sqrt(error_norms ratio): ||A - U S V||_F / ||A||_F on the device."""
    e2, a2 = error_norms(ctx, spec, comp, rows)
    return (e2 / a2) ** 0.5 if a2 > 0 else 0.0


def set_jacobi_groups(g):
    """hbaca_debug_set_jacobi_groups: clusters per core for the Jacobi SVD of
    cores too large for one cluster (0 = automatic, 1 = one); returns the
    previous setting."""
    return int(lib().hbaca_debug_set_jacobi_groups(int(g)))


def set_qr_groups(g):
    """hbaca_debug_set_qr_groups: upper bound on the clusters per matrix of
    the QR / Q application of stages with few matrices (0 = automatic);
    returns the previous setting."""
    return int(lib().hbaca_debug_set_qr_groups(int(g)))


def set_qr_cluster(c):
    """hbaca_debug_set_qr_cluster: CTAs per matrix of the QR and Q-application
    launches of later calls (0 = per-stage choice); returns the previous
    setting."""
    return int(lib().hbaca_debug_set_qr_cluster(int(c)))


def set_jacobi_cluster(c):
    """hbaca_debug_set_jacobi_cluster: Jacobi CTAs per core of later calls (0 =
    per-stage choice); returns the previous setting."""
    return int(lib().hbaca_debug_set_jacobi_cluster(int(c)))


def set_jacobi_sweeps(n):
    """hbaca_debug_set_jacobi_sweeps: Jacobi sweep cap of later calls (0 =
    default); returns the previous cap."""
    return int(lib().hbaca_debug_set_jacobi_sweeps(int(n)))


class Compressed:
    """Output of compress(): U (m x r), S (r), V (r x n) as torch views, plus the
    workspace (which holds the leaf tapes)."""

    def __init__(self, U, S, V, rank, ws, res):
        self.U, self.S, self.V, self.rank, self.ws, self.res = U, S, V, rank, ws, res


_WS_CHECKED = {}


def _check_workspace(ws, need_fn, key):
    """The library cannot see the size of a caller's buffer: refuse a
    workspace smaller than the plan of these arguments needs (the answer is
    cached per argument bytes and buffer)."""
    k = key + (ws.data_ptr(), ws.numel() * ws.element_size())
    if k in _WS_CHECKED:
        return
    need = need_fn()
    have = ws.numel() * ws.element_size()
    if not ws.is_cuda or have < need:
        raise HbacaError(7, "workspace of %d bytes; these arguments need %d" % (have, need))
    if len(_WS_CHECKED) > 4096:
        _WS_CHECKED.clear()
    _WS_CHECKED[k] = True


def _check_out(Ut, S, V, cap, m, n, dt):
    """Caller-provided output buffers must hold cap x m, cap and cap x n."""
    ok = (Ut.is_cuda and S.is_cuda and V.is_cuda and Ut.dtype == dt and V.dtype == dt and S.dtype == _torch().float64
          and Ut.is_contiguous() and V.is_contiguous() and S.is_contiguous()
          and Ut.numel() >= cap * m and S.numel() >= cap and V.numel() >= cap * n)
    if not ok:
        raise HbacaError(1, "output buffers must be contiguous device tensors of %d x %d, %d and %d x %d" % (cap, m, cap, cap, n))


def _torch():
    import torch
    return torch


def compress(ctx, spec, opts, stream=None, ws=None, out=None):
    """hbaca_compress on the current torch stream.  ``ws`` / ``out`` may be
    passed to reuse device buffers across calls."""
    import torch
    m, n = spec.m, spec.n
    cap = opts.rank_cap if opts.rank_cap else min(m, n, 1024)
    dt = torch.complex128 if spec.complex else torch.float64
    if ws is None:
        ws = torch.empty(workspace_size(spec.gen, opts), dtype=torch.uint8, device="cuda")
    else:
        _check_workspace(ws, lambda: workspace_size(spec.gen, opts), (bytes(spec.gen), bytes(opts)))
    if out is None:
        Ut = torch.empty((cap, m), dtype=dt, device="cuda")
        S = torch.empty(cap, dtype=torch.float64, device="cuda")
        V = torch.empty((cap, n), dtype=dt, device="cuda")
    else:
        Ut, S, V = out
        _check_out(Ut, S, V, min(cap, m, n), m, n, dt)
    res = Result(U=Ut.data_ptr(), ldu=m, S=S.data_ptr(), V=V.data_ptr(), ldv=n)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib().hbaca_compress(ctx.ptr, ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.byref(res),
                               ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(stream)))
    r = _host_rank(res, opts)
    c = Compressed(Ut[:r].T, S[:r], V[:r], r, ws, res)
    c.buffers = (Ut, S, V)
    return c


def compress_noalloc(ctx, spec, opts, stream=None, out=None):
    """hbaca_compress_noalloc: the library's built-in workspace (the call
    itself allocates no device memory; ``out`` buffers are the caller's)."""
    import torch
    m, n = spec.m, spec.n
    cap = opts.rank_cap if opts.rank_cap else min(m, n, 1024)
    dt = torch.complex128 if spec.complex else torch.float64
    if out is None:
        out = (torch.empty((cap, m), dtype=dt, device="cuda"), torch.empty(cap, dtype=torch.float64, device="cuda"),
               torch.empty((cap, n), dtype=dt, device="cuda"))
    Ut, S, V = out
    res = Result(U=Ut.data_ptr(), ldu=m, S=S.data_ptr(), V=V.data_ptr(), ldv=n)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib().hbaca_compress_noalloc(ctx.ptr, ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.byref(res),
                                       ctypes.c_void_p(stream)))
    r = _host_rank(res, opts)
    c = Compressed(Ut[:r].T, S[:r], V[:r], r, None, res)
    c.buffers = out
    return c


def _colmajor(X, rows):
    """A (rows, nrhs) torch float64 CUDA tensor as a column-major buffer:
    returns (buffer tensor of shape (nrhs, rows), ld)."""
    import torch
    Xt = X.detach().to(device="cuda", dtype=torch.float64)
    if Xt.dim() == 1:
        Xt = Xt[:, None]
    assert Xt.shape[0] == rows
    return Xt.t().contiguous(), rows


def apply(ctx, spec, comp, X, stream=None):
    """Y = U diag(S) V X (hbaca_apply); X (n, nrhs) -> Y (m, nrhs), float64."""
    import torch
    Xc, ldx = _colmajor(X, spec.n)
    nrhs = Xc.shape[0]
    Yc = torch.empty((nrhs, spec.m), dtype=torch.float64, device="cuda")
    ws = torch.empty(lib().hbaca_apply_workspace_size(max(comp.rank, 1), nrhs), dtype=torch.uint8, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib().hbaca_apply(ctx.ptr, ctypes.byref(spec.gen), ctypes.byref(comp.res), ctypes.c_void_p(Xc.data_ptr()),
                            nrhs, ldx, ctypes.c_void_p(Yc.data_ptr()), spec.m, ctypes.c_void_p(ws.data_ptr()),
                            ctypes.c_void_p(stream)))
    return Yc.t()


def apply_backward(ctx, spec, opts, comp, X, dY, stream=None, want_dX=True, keep_workspace=False):
    """hbaca_apply_backward: (d_h, d_x, d_y, dX) for Y = (U diag(S) V) X with
    the forward's pivots and ranks frozen (the forward must have run with
    FLAG_TAPE; ``comp`` is its result)."""
    import torch
    Xc, ldx = _colmajor(X, spec.n)
    dYc, lddy = _colmajor(dY, spec.m)
    nrhs = Xc.shape[0]
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = ctypes.c_void_p(stream)
    nb = lib().hbaca_backward_workspace_size(ctypes.byref(spec.gen), ctypes.byref(opts),
                                             ctypes.c_void_p(comp.ws.data_ptr()), nrhs, st)
    if nb == 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    bws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dh = torch.empty(1, dtype=torch.float64, device="cuda")
    dx = torch.empty((spec.m, spec.gen.dim), dtype=torch.float64, device="cuda")
    dy = torch.empty((spec.n, spec.gen.dim), dtype=torch.float64, device="cuda")
    dXc = torch.empty((nrhs, spec.n), dtype=torch.float64, device="cuda") if want_dX else None
    check(lib().hbaca_apply_backward(ctx.ptr, ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.byref(comp.res),
                                     ctypes.c_void_p(comp.ws.data_ptr()), ctypes.c_void_p(Xc.data_ptr()), nrhs, ldx,
                                     ctypes.c_void_p(dYc.data_ptr()), lddy, ctypes.c_void_p(dh.data_ptr()),
                                     ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dy.data_ptr()),
                                     ctypes.c_void_p(dXc.data_ptr() if want_dX else None), spec.n,
                                     ctypes.c_void_p(bws.data_ptr()), nb, st))
    if keep_workspace:
        return dh[0], dx, dy, (dXc.t() if want_dX else None), bws
    return dh[0], dx, dy, (dXc.t() if want_dX else None)


def apply_backward_batched(batch, Xs, dYs, stream=None, want_dX=True):
    """hbaca_apply_backward_batched for a Batch compressed with FLAG_TAPE:
    Xs[b] (n_b, nrhs), dYs[b] (m_b, nrhs).  Returns (d_h (nblocks,), [d_x_b],
    [d_y_b], [dX_b])."""
    import torch
    nb = len(batch.specs)
    Xc = [_colmajor(X, s.n)[0] for X, s in zip(Xs, batch.specs)]
    dYc = [_colmajor(dY, s.m)[0] for dY, s in zip(dYs, batch.specs)]
    nrhs = Xc[0].shape[0]
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = ctypes.c_void_p(stream)
    nbytes = lib().hbaca_backward_workspace_size_batched(nb, batch.gens, ctypes.byref(batch.opts),
                                                         ctypes.c_void_p(batch.ws.data_ptr()), nrhs, st)
    if nbytes == 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    bws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dh = torch.empty(nb, dtype=torch.float64, device="cuda")
    dx = [torch.empty((s.m, s.gen.dim), dtype=torch.float64, device="cuda") for s in batch.specs]
    dy = [torch.empty((s.n, s.gen.dim), dtype=torch.float64, device="cuda") for s in batch.specs]
    dX = [torch.empty((nrhs, s.n), dtype=torch.float64, device="cuda") for s in batch.specs] if want_dX else None
    ptrs = lambda ts: (ctypes.c_void_p * nb)(*[t.data_ptr() for t in ts])
    check(lib().hbaca_apply_backward_batched(batch.ctx.ptr, nb, batch.gens, ctypes.byref(batch.opts), batch.res,
                                             ctypes.c_void_p(batch.ws.data_ptr()), ptrs(Xc), nrhs, ptrs(dYc),
                                             ctypes.c_void_p(dh.data_ptr()), ptrs(dx), ptrs(dy),
                                             ptrs(dX) if want_dX else None, ctypes.c_void_p(bws.data_ptr()), nbytes,
                                             st))
    return dh, dx, dy, ([t.t() for t in dX] if want_dX else None)


def _autograd_function():
    import torch

    class GaussianHBACAApply(torch.autograd.Function):
        """Y = A_hat(h, x, y) X where A_hat = U diag(S) V is the H-BACA
        compression (Alg. 3) of the Gaussian kernel matrix
        exp(-||x_i - y_j||^2 / (2 h^2)); the backward differentiates A_hat with
        the forward's pivots and truncation ranks frozen."""

        @staticmethod
        def forward(fctx, h, x, y, X, hctx, eps, d, levels, seed, rank_cap, leaf_rank_cap):
            spec = gaussian(x, y, float(h))
            opts = make_opts(eps, d, levels, seed=seed, rank_cap=rank_cap, leaf_rank_cap=leaf_rank_cap,
                             flags=FLAG_TAPE)
            comp = compress(hctx, spec, opts)
            Y = apply(hctx, spec, comp, X)
            fctx.state = (hctx, spec, opts, comp)
            fctx.save_for_backward(X)
            return Y

        @staticmethod
        def backward(fctx, dY):
            hctx, spec, opts, comp = fctx.state
            (X,) = fctx.saved_tensors
            dh, dx, dy, dX = apply_backward(hctx, spec, opts, comp, X, dY.contiguous())
            return dh.reshape(()), dx, dy, dX, None, None, None, None, None, None, None

    return GaussianHBACAApply


_AUTOGRAD = None


def gaussian_hbaca_apply(h, x, y, X, ctx, eps, d, levels, seed=0, rank_cap=0, leaf_rank_cap=0):
    """Differentiable Y = A_hat(h, x, y) X (torch.autograd), see GaussianHBACAApply."""
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _autograd_function()
    return _AUTOGRAD.apply(h, x, y, X, ctx, eps, d, levels, seed, rank_cap, leaf_rank_cap)


def _trace_call(call, d, max_iters):
    """Run a trace-reading call with fresh host arrays; returns the record dict."""
    import numpy as np
    I = np.full(max_iters * d, -1, np.int32)
    J = np.full(max_iters * d, -1, np.int32)
    jb = np.full(max_iters * d, -1, np.int32)
    dI = np.zeros(max_iters, np.int32)
    dJ = np.zeros(max_iters, np.int32)
    dk = np.zeros(max_iters, np.int32)
    nu = np.zeros(max_iters)
    mu = np.zeros(max_iters)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    tr = LeafTrace(max_iters=max_iters, d=d, I=p(I), J=p(J), jbar=p(jb), dI=p(dI), dJ=p(dJ), dk=p(dk),
                   nu=p(nu), mu=p(mu))
    check(call(tr))
    recs = []
    for k in range(tr.iters):
        recs.append(dict(I=list(I[k * d:k * d + dI[k]]), J=list(J[k * d:k * d + dJ[k]]),
                         jbar=list(jb[k * d:k * d + dk[k]]), dk=int(dk[k]), nu=float(nu[k]), mu=float(mu[k])))
    return dict(iters=tr.iters, rank_baca=tr.rank_baca, rank=tr.rank, stop=STOP.get(tr.stop, tr.stop), trace=recs)


def _gen_array(specs):
    arr = (Gen * len(specs))()
    for i, s in enumerate(specs):
        arr[i] = s.gen
    return arr


class Batch:
    """A batched call set up once: the host arrays of generators and results,
    the workspace and the per-block output buffers, so that repeated calls
    (timing, training loops) do no Python-side work but the ABI call."""

    def __init__(self, ctx, specs, opts, ws=None):
        import torch
        self.ctx, self.specs, self.opts = ctx, list(specs), opts
        n = len(self.specs)
        self.gens = _gen_array(self.specs)
        if ws is None:
            # with an automatic leaf cluster size, room for every size the
            # autotuner may try (the plans differ by their scratch)
            sizes = [opts.cluster] + ([1, 2, 4, 8, 16] if opts.cluster == 0 else [])
            nbytes = 0
            for c in sizes:
                o = Opts.from_buffer_copy(opts)
                o.cluster = c
                nb = lib().hbaca_workspace_size_batched(n, self.gens, ctypes.byref(o))
                if nb == 0 and c == sizes[0]:
                    raise HbacaError(1, lib().hbaca_last_error().decode())
                nbytes = max(nbytes, nb)
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.ws = ws
        self.res = (Result * n)()
        self.bufs = []
        for i, s in enumerate(self.specs):
            cap = min(opts.rank_cap, s.m, s.n) if opts.rank_cap else min(s.m, s.n, 1024)
            dt = torch.complex128 if s.complex else torch.float64
            Ut = torch.empty((cap, s.m), dtype=dt, device="cuda")
            S = torch.empty(cap, dtype=torch.float64, device="cuda")
            V = torch.empty((cap, s.n), dtype=dt, device="cuda")
            self.res[i] = Result(U=Ut.data_ptr(), ldu=s.m, S=S.data_ptr(), V=V.data_ptr(), ldv=s.n)
            self.bufs.append((Ut, S, V))

    def run(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        n = len(self.specs)
        _check_workspace(self.ws, lambda: lib().hbaca_workspace_size_batched(n, self.gens, ctypes.byref(self.opts)),
                         (bytes(self.gens), bytes(self.opts)))
        check(lib().hbaca_compress_batched(self.ctx.ptr, len(self.specs), self.gens, ctypes.byref(self.opts),
                                           self.res, ctypes.c_void_p(self.ws.data_ptr()),
                                           ctypes.c_void_p(stream)))
        return self

    def autotune(self, stream=None):
        """hbaca_autotune_batched on this batch's workspace: sets opts.cluster
        to the fastest leaf cluster size and returns (cluster, ms)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        c = ctypes.c_int32(0)
        ms = ctypes.c_double(0.0)
        check(lib().hbaca_autotune_batched(self.ctx.ptr, len(self.specs), self.gens, ctypes.byref(self.opts),
                                           ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                           ctypes.c_void_p(stream), ctypes.byref(c), ctypes.byref(ms)))
        self.opts.cluster = c.value
        return c.value, ms.value

    def ranks(self):
        return [int(self.res[i].rank) for i in range(len(self.specs))]

    def results(self):
        out = []
        for i in range(len(self.specs)):
            r = int(self.res[i].rank)
            Ut, S, V = self.bufs[i]
            c = Compressed(Ut[:r].T, S[:r], V[:r], r, self.ws, self.res[i])
            c.buffers = self.bufs[i]
            out.append(c)
        return out


def compress_batched(ctx, specs, opts, ws=None, stream=None):
    """hbaca_compress_batched over a list of GenSpec (one per block); returns a
    list of Compressed (one per block) sharing the workspace."""
    return Batch(ctx, specs, opts, ws).run(stream).results()


def read_leaf_trace_batched(specs, opts, ws, block, leaf, max_iters=4096):
    import torch
    gens = _gen_array(specs)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _trace_call(lambda tr: lib().hbaca_read_leaf_trace_batched(len(specs), gens, ctypes.byref(opts),
                                                                       ctypes.c_void_p(ws.data_ptr()), block, leaf,
                                                                       ctypes.byref(tr), st), opts.d, max_iters)


def read_leaf_trace(spec, opts, ws, leaf, max_iters=4096):
    """Per-leaf BACA record of the last single-block compress into `ws`."""
    import torch
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _trace_call(lambda tr: lib().hbaca_read_leaf_trace(ctypes.byref(spec.gen), ctypes.byref(opts),
                                                              ctypes.c_void_p(ws.data_ptr()), leaf,
                                                              ctypes.byref(tr), st), opts.d, max_iters)


def read_block(spec, opts, ws, store, level, block):
    """Intermediate block (store 0: after the vertical merge of ``level``, level
    0 = re-compressed leaves; store 1: after the horizontal merge of ``level``)
    as numpy U (m x r), S (r), V (r x n)."""
    import numpy as np
    import torch
    m, n = spec.m, spec.n
    cap = opts.rank_cap if opts.rank_cap else min(m, n, 1024)
    dt = np.complex128 if spec.complex else np.float64
    # block sizes are at most the matrix sizes
    Ub = np.zeros(m * cap, dt)
    Sb = np.zeros(cap)
    Vb = np.zeros(cap * n, dt)
    mo, no, ro, co = (ctypes.c_int64() for _ in range(4))
    check(lib().hbaca_debug_read_block(ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()),
                                       store, level, block, Ub.ctypes.data_as(ctypes.c_void_p),
                                       Sb.ctypes.data_as(ctypes.c_void_p), Vb.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(mo), ctypes.byref(no), ctypes.byref(ro), ctypes.byref(co),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    bm, bn, r = mo.value, no.value, ro.value
    U = Ub[:bm * r].reshape(r, bm).T
    V = Vb[:r * bn].reshape(r, bn)
    return U, Sb[:r], V


def kdtree_order(points, leaf):
    """hbaca_kdtree_order: a permutation (numpy int64) ordering the points so
    that every H-BACA index-tree node down to `leaf` points is a KD cell."""
    import numpy as np
    P = np.ascontiguousarray(np.asarray(points, np.float64))
    perm = np.empty(P.shape[0], np.int64)
    check(lib().hbaca_kdtree_order(P.ctypes.data_as(ctypes.c_void_p), P.shape[0], P.shape[1], int(leaf),
                                   perm.ctypes.data_as(ctypes.c_void_p)))
    return perm


def hmatrix_blocks(x, y, leaf, eta):
    """hbaca_hmatrix_blocks for ordered point sets x, y: an (nblocks, 5) int64
    array of (row start, rows, column start, columns, admissible)."""
    import numpy as np
    X = np.ascontiguousarray(np.asarray(x, np.float64))
    Y = np.ascontiguousarray(np.asarray(y, np.float64))
    args = (X.ctypes.data_as(ctypes.c_void_p), X.shape[0], Y.ctypes.data_as(ctypes.c_void_p), Y.shape[0],
            X.shape[1], int(leaf), float(eta))
    n = lib().hbaca_hmatrix_blocks(*args, None, 0)
    if n < 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    out = np.empty((n, 5), np.int64)
    lib().hbaca_hmatrix_blocks(*args, out.ctypes.data_as(ctypes.c_void_p), n)
    return out


def read_leaf_factors(spec, opts, ws, leaf, m_leaf, n_leaf):
    """BACA factors (U m_leaf x r, V r x n_leaf) of one leaf of a taped call."""
    import numpy as np
    import torch
    cap = min(m_leaf, n_leaf, 1024)
    dt = np.complex128 if spec.complex else np.float64
    Ub = np.zeros(m_leaf * cap, dt)
    Vb = np.zeros(cap * n_leaf, dt)
    mo, no, ro = (ctypes.c_int64() for _ in range(3))
    check(lib().hbaca_debug_read_leaf_factors(ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()),
                                              leaf, Ub.ctypes.data_as(ctypes.c_void_p), Vb.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(mo), ctypes.byref(no), ctypes.byref(ro),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    r = ro.value
    return Ub[:mo.value * r].reshape(r, mo.value).T, Vb[:r * no.value].reshape(r, no.value)


def plan_json(spec, opts):
    """Workspace layout of (spec, opts) as a dict (debugging aid)."""
    import json
    n = lib().hbaca_debug_plan_json(ctypes.byref(spec.gen), ctypes.byref(opts), None, 0)
    buf = ctypes.create_string_buffer(n)
    lib().hbaca_debug_plan_json(ctypes.byref(spec.gen), ctypes.byref(opts), buf, n)
    return json.loads(buf.value.decode())


def backward_json(spec, opts, ws, nrhs):
    """Layout of the reverse pass (debugging aid), as a dict."""
    import json
    import torch
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = lib().hbaca_debug_backward_json(ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()),
                                        nrhs, None, 0, st)
    if n < 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    buf = ctypes.create_string_buffer(int(n))
    lib().hbaca_debug_backward_json(ctypes.byref(spec.gen), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()), nrhs,
                                    buf, n, st)
    return json.loads(buf.value.decode())


KERNEL_CLASSES = ["baca_leaf_kernel", "pack_kernel", "qr_kernel", "core_kernel", "qrcp_core_kernel",
                  "jacobi_kernel", "finish_kernel", "qapply_kernel", "blockprod_kernel", "copyroot_kernel"]


def kernel_times(ctx):
    """{kernel: (ms, launches)} of the last profiled call (CUDA events)."""
    ms = (ctypes.c_double * len(KERNEL_CLASSES))()
    nl = (ctypes.c_int32 * len(KERNEL_CLASSES))()
    check(lib().hbaca_kernel_times(ctx.ptr, ms, nl))
    return {k: (ms[i], nl[i]) for i, k in enumerate(KERNEL_CLASSES)}


def launch_times(ctx):
    """Per launch of the last profiled call: list of (kernel class name, stage,
    start ms, ms)."""
    import numpy as np
    n = lib().hbaca_debug_launch_times(ctx.ptr, None, None, None, None, 0)
    if n < 0:
        raise HbacaError(1, lib().hbaca_last_error().decode())
    cls = np.zeros(n, np.int32)
    stg = np.zeros(n, np.int32)
    t0 = np.zeros(n)
    ms = np.zeros(n)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib().hbaca_debug_launch_times(ctx.ptr, p(cls), p(stg), p(t0), p(ms), n)
    return [(KERNEL_CLASSES[c], int(s), float(a), float(b)) for c, s, a, b in zip(cls, stg, t0, ms)]


def phase_times(ctx):
    """(ms BACA, ms leaf re-compression, ms merges, ms total), launches of the
    last call made with FLAG_PROFILE."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int32()
    check(lib().hbaca_phase_times(ctx.ptr, ms, ctypes.byref(n)))
    return tuple(ms), n.value


PROBE_PATH = os.path.join(HERE, "libhbaca_probe.so")
PROBE_SIGNATURES = [
    ("hbaca_debug_fp64_probe", ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
]
_PROBE = None


def probe_lib():
    """Load libhbaca_probe.so, the FP64 unit-rate probe the benchmark reports."""
    global _PROBE
    if _PROBE is None:
        if not os.path.exists(PROBE_PATH):
            raise RuntimeError("libhbaca_probe.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(PROBE_PATH)
        for name, res, args in PROBE_SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _PROBE = L
    return _PROBE


def fp64_probe():
    """(DFMA, DMMA) TFLOP/s measured on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(probe_lib().hbaca_debug_fp64_probe(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value
