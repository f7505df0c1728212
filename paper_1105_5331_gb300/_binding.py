"""Thin ctypes binding over the C ABI in ``include/cp.h``.

Argument marshalling only: every computation runs in the CUDA library
``libcp_gb300.so``.  The functions keep the C names.  Array arguments may be
torch tensors (their ``data_ptr()`` is passed; device tensors for device
arguments), numpy arrays (host arguments only) or raw integer addresses.
If the library is missing, importing this module raises ImportError: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcp_gb300.so")

CP_FP64 = 0
CP_MIXED_BF16X3 = 1
CP_DTYPE_F32 = 0
CP_DTYPE_F64 = 1

STATUS_NAMES = {
    0: "CP_OK", 1: "CP_ERR_ARG", 2: "CP_ERR_SHAPE", 3: "CP_ERR_OOM", 4: "CP_ERR_CUDA",
    5: "CP_ERR_NOT_SPD", 6: "CP_ERR_NONFINITE", 7: "CP_ERR_LINESEARCH", 8: "CP_ERR_MAXIT",
    9: "CP_ERR_TIMEOUT", 10: "CP_ERR_BUSY", 11: "CP_ERR_UNSUPPORTED",
}

# Every symbol include/cp.h declares (checked by the tests).
EXPORTED = [
    "cp_ctx_create", "cp_ctx_destroy", "cp_last_error", "cp_ctx_sync", "cp_ctx_stream",
    "cp_kernel_launches", "cp_ctx_timer_enable", "cp_ctx_timer_read",
    "cp_tensor_dense", "cp_tensor_coo", "cp_tensor_info", "cp_tensor_sorted_mode",
    "cp_tensor_destroy", "cp_mttkrp", "cp_mttkrp_variants", "cp_mttkrp_noalloc", "cp_mttkrp_dimtree", "cp_fg", "cp_als_sweep", "cp_normalize",
    "ngmres_step",
    "cp_ls_opts_default", "linesearch", "cp_solve_opts_default", "cp_solve",
    "cp_solve_batch", "cp_solve_many", "cp_many_set_round", "cp_many_plan", "cp_server_create", "cp_server_submit", "cp_server_poll", "cp_server_cancel",
    "cp_server_drain", "cp_server_stats", "cp_server_set_engine", "cp_server_destroy",
]


class CpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cp_ls_opts(C.Structure):
    _fields_ = [("ftol", C.c_double), ("gtol", C.c_double), ("xtol", C.c_double),
                ("stpmin", C.c_double), ("stpmax", C.c_double), ("stp0", C.c_double),
                ("maxfev", C.c_int)]


class cp_solve_opts(C.Structure):
    _fields_ = [("R", C.c_int), ("w", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("eps", C.c_double), ("prec", C.c_int), ("polish", C.c_int),
                ("mixed_tol_factor", C.c_double), ("ls", cp_ls_opts),
                ("mixed_maxfev", C.c_int), ("dimtree", C.c_int), ("mixed_stall", C.c_int),
                ("mixed_min_entries", C.c_int)]


class cp_solve_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("fg_evals", C.c_int), ("als_sweeps", C.c_int),
                ("restarts", C.c_int), ("ls_failures", C.c_int), ("converged", C.c_int),
                ("mixed_iters", C.c_int), ("fp64_iters", C.c_int),
                ("f", C.c_double), ("gnorm_over_P", C.c_double), ("normT2", C.c_double),
                ("t_total_s", C.c_double), ("ls_trials", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(this package has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I, I64, D, VP = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_void_p
    sig = {
        "cp_ctx_create": (I, [I, VP, C.POINTER(VP)]),
        "cp_ctx_destroy": (None, [VP]),
        "cp_last_error": (C.c_char_p, []),
        "cp_ctx_sync": (I, [VP]),
        "cp_ctx_stream": (VP, [VP]),
        "cp_kernel_launches": (C.c_ulonglong, []),
        "cp_ctx_timer_enable": (I, [VP, I]),
        "cp_ctx_timer_read": (I, [VP, I, C.POINTER(D), C.POINTER(I)]),
        "cp_tensor_dense": (I, [VP, I, P, I, VP, C.POINTER(VP)]),
        "cp_tensor_coo": (I, [VP, I, P, I64, VP, VP, C.POINTER(VP)]),
        "cp_tensor_info": (I, [VP, C.POINTER(I), P, C.POINTER(D)]),
        "cp_tensor_sorted_mode": (I, [VP, VP, I, P, P, P, C.POINTER(I64)]),
        "cp_tensor_destroy": (None, [VP]),
        "cp_mttkrp": (I, [VP, VP, I, VP, I, VP, I]),
        "cp_mttkrp_noalloc": (I, [VP, VP, I, VP, I, VP]),
        "cp_mttkrp_dimtree": (I, [VP, VP, I, VP, I, VP, I]),
        "cp_mttkrp_variants": (I, [VP, VP, I, VP, VP, P, I, VP, I]),
        "cp_fg": (I, [VP, VP, I, VP, VP, VP, I]),
        "cp_als_sweep": (I, [VP, VP, I, VP, I, I]),
        "cp_normalize": (I, [VP, I, P, I, VP, VP, VP]),
        "ngmres_step": (I, [VP, I64, I, VP, VP, VP, VP, D, VP, VP]),
        "cp_ls_opts_default": (None, [C.POINTER(cp_ls_opts)]),
        "linesearch": (I, [VP, VP, I, VP, D, VP, VP, C.POINTER(cp_ls_opts), VP, C.POINTER(D), VP,
                           C.POINTER(D), C.POINTER(I), C.POINTER(I), I]),
        "cp_solve_opts_default": (None, [C.POINTER(cp_solve_opts), I]),
        "cp_solve": (I, [VP, VP, C.POINTER(cp_solve_opts), VP, C.POINTER(cp_solve_report)]),
        "cp_solve_batch": (I, [VP, I, C.POINTER(VP), C.POINTER(cp_solve_opts), C.POINTER(VP),
                               C.POINTER(cp_solve_report)]),
        "cp_solve_many": (I, [VP, I, C.POINTER(VP), C.POINTER(cp_solve_opts), C.POINTER(VP),
                              C.POINTER(cp_solve_report), I]),
        "cp_many_plan": (I, [VP, VP, C.POINTER(cp_solve_opts), VP, C.POINTER(I)]),
        "cp_many_set_round": (I, [VP, D]),
        "cp_server_create": (I, [VP, C.c_size_t, I, C.POINTER(VP)]),
        "cp_server_submit": (I, [VP, I, P, I, VP, C.POINTER(cp_solve_opts), VP, VP, C.POINTER(C.c_uint64)]),
        "cp_server_poll": (I, [VP, C.c_uint64, C.POINTER(I), C.POINTER(I), C.POINTER(cp_solve_report),
                               C.POINTER(D)]),
        "cp_server_cancel": (I, [VP, C.c_uint64]),
        "cp_server_drain": (I, [VP, D]),
        "cp_server_stats": (I, [VP, C.POINTER(D), C.POINTER(D), C.POINTER(D), C.POINTER(I),
                                C.POINTER(C.c_size_t)]),
        "cp_server_set_engine": (I, [VP, I, C.c_longlong, I]),
        "cp_server_destroy": (None, [VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def library():
    return _lib


def _check(status: int, allow=()):
    if status != 0 and status not in allow:
        raise CpError(status, (_lib.cp_last_error() or b"").decode())
    return status


def _ptr(x):
    """Address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("array arguments must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as an array")


def _dims(dims):
    arr = (C.c_int64 * len(dims))(*[int(d) for d in dims])
    return arr


class Ctx:
    """Owning wrapper of a cp_ctx*."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            _lib.cp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tensor:
    """Owning wrapper of a cp_tensor*."""

    def __init__(self, handle, dims, kind):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.kind = kind

    def close(self):
        if self.handle:
            _lib.cp_tensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(x):
    return x.handle if hasattr(x, "handle") else x


CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy


def cp_ctx_create(device: int = 0, stream=None) -> Ctx:
    """Context on ``device``.  ``stream``: None creates a private stream; a
    torch stream (or raw handle) is borrowed.  Torch's default stream has
    handle 0, which C reads as "none", so it is passed as cudaStreamLegacy to
    keep the library ordered with torch's work."""
    out = C.c_void_p()
    s = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    if stream is not None and s == 0:
        s = CUDA_STREAM_LEGACY
    _check(_lib.cp_ctx_create(int(device), s, C.byref(out)))
    return Ctx(out.value)


def cp_ctx_destroy(ctx):
    ctx.close() if hasattr(ctx, "close") else _lib.cp_ctx_destroy(ctx)


def cp_last_error() -> str:
    return (_lib.cp_last_error() or b"").decode()


def cp_ctx_sync(ctx):
    return _check(_lib.cp_ctx_sync(_h(ctx)))


def cp_ctx_stream(ctx) -> int:
    return _lib.cp_ctx_stream(_h(ctx))


def cp_kernel_launches() -> int:
    return int(_lib.cp_kernel_launches())


TIMER_TC, TIMER_F64, TIMER_COO = 0, 1, 2


def cp_ctx_timer_enable(ctx, enable: bool = True):
    _check(_lib.cp_ctx_timer_enable(_h(ctx), int(bool(enable))))


def cp_ctx_timer_read(ctx, which: int):
    """(total_ms, launches) of one MTTKRP kernel family since enabling."""
    ms = C.c_double()
    n = C.c_int()
    _check(_lib.cp_ctx_timer_read(_h(ctx), int(which), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def cp_tensor_dense(ctx, data, dims=None, dtype=None) -> Tensor:
    """Dense tensor from a torch tensor / numpy array (float32 or float64)."""
    if dims is None:
        dims = tuple(data.shape)
    if dtype is None:
        name = str(data.dtype)
        dtype = CP_DTYPE_F64 if "float64" in name else CP_DTYPE_F32
    out = C.c_void_p()
    _check(_lib.cp_tensor_dense(_h(ctx), len(dims), _dims(dims), int(dtype), _ptr(data), C.byref(out)))
    return Tensor(out.value, dims, "dense")


def cp_tensor_coo(ctx, dims, coords, vals) -> Tensor:
    nnz = int(coords.shape[0])
    out = C.c_void_p()
    _check(_lib.cp_tensor_coo(_h(ctx), len(dims), _dims(dims), nnz, _ptr(coords) if nnz else None,
                              _ptr(vals) if nnz else None, C.byref(out)))
    t = Tensor(out.value, dims, "coo")
    t.nnz = nnz
    return t


def cp_tensor_info(t):
    N = C.c_int()
    dims = (C.c_int64 * 8)()
    n2 = C.c_double()
    _check(_lib.cp_tensor_info(_h(t), C.byref(N), dims, C.byref(n2)))
    return N.value, tuple(dims[: N.value]), n2.value


def cp_tensor_sorted_mode(ctx, t, mode: int):
    import numpy as np
    nseg = C.c_int64()
    _check(_lib.cp_tensor_sorted_mode(_h(ctx), _h(t), int(mode), None, None, None, C.byref(nseg)))
    N, dims, _ = cp_tensor_info(t)
    nnz = getattr(t, "nnz", None)
    perm = np.empty(nnz if nnz is not None else 0, dtype=np.int64)
    seg_ptr = np.empty(nseg.value + 1, dtype=np.int64)
    seg_row = np.empty(nseg.value, dtype=np.int64)
    _check(_lib.cp_tensor_sorted_mode(_h(ctx), _h(t), int(mode), _ptr(perm) if perm.size else None,
                                      _ptr(seg_ptr), _ptr(seg_row) if seg_row.size else None,
                                      C.byref(nseg)))
    return perm, seg_ptr, seg_row


def cp_tensor_destroy(t):
    t.close() if hasattr(t, "close") else _lib.cp_tensor_destroy(t)


def cp_mttkrp(ctx, t, R: int, u, mode: int, out, prec: int = CP_FP64):
    _check(_lib.cp_mttkrp(_h(ctx), _h(t), int(R), _ptr(u), int(mode), _ptr(out), int(prec)))
    return out


def cp_mttkrp_variants(ctx, t, R: int, u, d, modes, out, prec: int = CP_FP64):
    """Khatri-Rao variant MTTKRPs along u + beta d for the listed modes; out
    holds, per mode in the order given, 2^(N-1) blocks of I_mode x R."""
    ms = (C.c_int * len(modes))(*[int(m) for m in modes])
    _check(_lib.cp_mttkrp_variants(_h(ctx), _h(t), int(R), _ptr(u), _ptr(d), ms, len(modes), _ptr(out),
                                   int(prec)))
    return out


def cp_mttkrp_dimtree(ctx, t, R: int, u, contracted: int, out, prec: int = 1):
    """W = T x_contracted A^(contracted), then the MTTKRPs of the other two
    modes from W (in increasing mode order, back to back in out)."""
    _check(_lib.cp_mttkrp_dimtree(_h(ctx), _h(t), int(R), _ptr(u), int(contracted), _ptr(out), int(prec)))


def cp_mttkrp_noalloc(ctx, t, R: int, u, mode: int, out):
    """FP64 dense MTTKRP that allocates no device memory (fixed 8 MiB library
    scratch shared by all calls; see include/cp.h)."""
    _check(_lib.cp_mttkrp_noalloc(_h(ctx), _h(t), int(R), _ptr(u), int(mode), _ptr(out)))
    return out


def cp_fg(ctx, t, R: int, u, f, g=None, prec: int = CP_FP64):
    _check(_lib.cp_fg(_h(ctx), _h(t), int(R), _ptr(u), _ptr(f), _ptr(g), int(prec)))


def cp_als_sweep(ctx, t, R: int, u, normalize: bool = False, prec: int = CP_FP64):
    _check(_lib.cp_als_sweep(_h(ctx), _h(t), int(R), _ptr(u), int(bool(normalize)), int(prec)))


def cp_normalize(ctx, dims, R: int, u, g=None, lam=None):
    _check(_lib.cp_normalize(_h(ctx), len(dims), _dims(dims), int(R), _ptr(u), _ptr(g), _ptr(lam)))


def ngmres_step(ctx, U, G, ubar, gbar, eps: float, uhat, alpha=None):
    m, P = int(U.shape[0]), int(U.shape[1])
    _check(_lib.ngmres_step(_h(ctx), P, m, _ptr(U), _ptr(G), _ptr(ubar), _ptr(gbar), float(eps),
                            _ptr(uhat), _ptr(alpha)))


def cp_ls_opts_default() -> cp_ls_opts:
    o = cp_ls_opts()
    _lib.cp_ls_opts_default(C.byref(o))
    return o


def linesearch(ctx, t, R: int, x0, f0: float, g0, d, x, g, opts: cp_ls_opts | None = None,
               prec: int = CP_FP64):
    """Returns (f, stp, nfev, info); x and g receive the final point and gradient."""
    f = C.c_double()
    stp = C.c_double()
    nfev = C.c_int()
    info = C.c_int()
    _check(_lib.linesearch(_h(ctx), _h(t), int(R), _ptr(x0), float(f0), _ptr(g0), _ptr(d),
                           C.byref(opts) if opts is not None else None, _ptr(x), C.byref(f), _ptr(g),
                           C.byref(stp), C.byref(nfev), C.byref(info), int(prec)))
    return f.value, stp.value, nfev.value, info.value


def cp_solve_opts_default(R: int) -> cp_solve_opts:
    o = cp_solve_opts()
    _lib.cp_solve_opts_default(C.byref(o), int(R))
    return o


def cp_solve(ctx, t, opts: cp_solve_opts, u) -> dict:
    """Runs the solve in place on u; returns the report as a dict.  A solve
    that stops at maxit is not an exception (report['converged'] == 0)."""
    rep = cp_solve_report()
    _check(_lib.cp_solve(_h(ctx), _h(t), C.byref(opts), _ptr(u), C.byref(rep)), allow=(8,))
    return rep.as_dict()


def cp_solve_batch(ctx, tensors, opts_list, us) -> list:
    """Solve several problems at once (each on its own stream); returns the
    reports.  A problem that stops at maxit is not an exception."""
    n = len(tensors)
    th = (C.c_void_p * n)(*[_h(t) for t in tensors])
    op = (cp_solve_opts * n)(*opts_list)
    up = (C.c_void_p * n)(*[_ptr(u) for u in us])
    reps = (cp_solve_report * n)()
    _check(_lib.cp_solve_batch(_h(ctx), n, th, op, up, reps), allow=(8,))
    return [r.as_dict() for r in reps]


def cp_solve_many(ctx, tensors, opts_list, us, cluster: int = 0) -> list:
    """Solve many small 3-way dense problems in one persistent launch (one
    thread-block cluster per problem at a time); returns the reports.  A
    problem that stops at maxit is not an exception."""
    n = len(tensors)
    th = (C.c_void_p * n)(*[_h(t) for t in tensors])
    op = (cp_solve_opts * n)(*opts_list)
    up = (C.c_void_p * n)(*[_ptr(u) for u in us])
    reps = (cp_solve_report * n)()
    _check(_lib.cp_solve_many(_h(ctx), n, th, op, up, reps, int(cluster)), allow=(8,))
    return [r.as_dict() for r in reps]


def cp_many_set_round(ctx, seconds: float):
    """Length of cp_solve_many's launches on this context (default 0.5 s)."""
    _check(_lib.cp_many_set_round(_h(ctx), float(seconds)))


def cp_many_plan(ctx, t, opts, u0) -> int:
    """Cluster size cp_solve_many gives this request's bucket (tuned on
    first use)."""
    out = C.c_int(0)
    _check(_lib.cp_many_plan(_h(ctx), _h(t), C.byref(opts), _ptr(u0), C.byref(out)))
    return out.value


class Server:
    """Owning wrapper of a cp_server*."""

    def __init__(self, handle):
        self.handle = handle
        self.buffers = []   # host arrays the worker reads or writes until the server is destroyed

    def close(self):
        if self.handle:
            _lib.cp_server_destroy(self.handle)
            self.handle = None
            self.buffers = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cp_server_create(ctx, hbm_budget_bytes: int, max_active: int) -> Server:
    out = C.c_void_p()
    _check(_lib.cp_server_create(_h(ctx), int(hbm_budget_bytes), int(max_active), C.byref(out)))
    return Server(out.value)


def cp_server_submit(server, data, opts: cp_solve_opts, u0, u_out) -> int:
    """data: host numpy array (float32/float64); u0, u_out: host float64 arrays."""
    dims = tuple(data.shape)
    dtype = CP_DTYPE_F64 if "float64" in str(data.dtype) else CP_DTYPE_F32
    rid = C.c_uint64()
    _check(_lib.cp_server_submit(_h(server), len(dims), _dims(dims), dtype, _ptr(data), C.byref(opts),
                                 _ptr(u0), _ptr(u_out), C.byref(rid)))
    if isinstance(server, Server):
        server.buffers.append(u_out)   # the result is written there later
    return rid.value


def cp_server_poll(server, req_id: int):
    """Returns None while running, else (status, report dict, latency_s)."""
    done = C.c_int()
    st = C.c_int()
    rep = cp_solve_report()
    lat = C.c_double()
    _check(_lib.cp_server_poll(_h(server), int(req_id), C.byref(done), C.byref(st), C.byref(rep), C.byref(lat)))
    if not done.value:
        return None
    return st.value, rep.as_dict(), lat.value


def cp_server_cancel(server, req_id: int):
    _check(_lib.cp_server_cancel(_h(server), int(req_id)))


def cp_server_drain(server, timeout_s: float = 600.0):
    _check(_lib.cp_server_drain(_h(server), float(timeout_s)))


def cp_server_stats(server) -> dict:
    p50, p99, sps = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int()
    peak = C.c_size_t()
    _check(_lib.cp_server_stats(_h(server), C.byref(p50), C.byref(p99), C.byref(sps), C.byref(n), C.byref(peak)))
    return {"p50_s": p50.value, "p99_s": p99.value, "solves_per_s": sps.value, "completed": n.value,
            "peak_bytes": peak.value}


def cp_server_set_engine(server, on: bool, max_work: int = 1 << 26, max_ctas: int = 0):
    """Route requests that fit the cluster engine and have at most max_work
    entries x R to it (on, the default), the rest to graph slots of their
    own; on=False: every request to a graph slot.  max_ctas: CTAs an engine
    round may use (0: as many as fit)."""
    _check(_lib.cp_server_set_engine(_h(server), 1 if on else 0, int(max_work), int(max_ctas)))


def cp_server_destroy(server):
    server.close() if hasattr(server, "close") else _lib.cp_server_destroy(server)
