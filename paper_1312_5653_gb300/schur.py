"""Python binding of libschur (include/schur.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; the arithmetic runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (float64, column-major multi-RHS
stored as shape (nrhs, ld)); the current torch CUDA stream is passed unless a stream is given.
If the compiled library is missing or fails to load, every call raises: there is no fallback.
"""
import ctypes
import os

from . import build as _build

SCHUR_OK = 0
SCHUR_EINVAL = -1
SCHUR_ENOMEM = -2
SCHUR_ENOTCONV = -3
SCHUR_EBREAKDOWN = -4
SCHUR_ETIMEOUT = -5
SCHUR_ECUDA = -6
SCHUR_EBUSY = -7
SCHUR_FP64 = 0
SCHUR_MIXED = 1
SCHUR_LOCAL_PER_SUBDOMAIN = 0
SCHUR_LOCAL_SHARED = 1
SCHUR_FACTOR_EXACT = 0
SCHUR_FACTOR_PW = 1


class schur_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nel", ctypes.c_int * 3)]


class schur_opts(ctypes.Structure):
    _fields_ = [("nsub", ctypes.c_int * 3), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("local_mode", ctypes.c_int), ("tc_split", ctypes.c_int), ("factor", ctypes.c_int),
                ("augment", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class schur_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_steps", ctypes.c_int), ("iters_total", ctypes.c_int),
                ("iters_first", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("ms_solve", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class schur_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_longlong), ("n_sub", ctypes.c_int), ("n_classes", ctypes.c_int),
                ("n_lambda", ctypes.c_int), ("n_coarse", ctypes.c_int), ("n_delta", ctypes.c_int),
                ("n_local", ctypes.c_int), ("bytes_operators", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class schur_kernel_time(ctypes.Structure):
    _fields_ = [("category", ctypes.c_int), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


class SchurError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d): %s" % (where, strerror(code), code, last_error()))


_lib = None
EXPORTS = [
    "schur_default_opts", "schur_setup", "schur_solve", "schur_solve_host", "schur_complex_solve",
    "schur_apply_mass", "schur_apply_stiffness", "schur_apply_S", "schur_kkt_apply", "schur_kkt_precond_apply",
    "schur_kkt_minres", "schur_partition", "schur_partition_export", "schur_get_info", "schur_ndof",
    "schur_destroy", "schur_strerror", "schur_last_error", "schur_debug_operator", "schur_profile_begin",
    "schur_profile_end", "schur_kernel_category_name", "schur_launch_count", "schur_apply_S_static", "schur_peak_probe", "schur_control_solve",
    "schur_server_default_opts", "schur_server_create", "schur_submit", "schur_poll", "schur_wait",
    "schur_server_info", "schur_server_destroy",
]


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libschur.so (building it first if it is missing and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libschur.so is not built: run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "schur_default_opts": (None, [ctypes.POINTER(schur_opts)]),
        "schur_setup": (I, [ctypes.POINTER(schur_mesh), D, ctypes.POINTER(schur_opts), P, ctypes.POINTER(P)]),
        "schur_solve": (I, [P, P, P, I, I, P, ctypes.POINTER(schur_stats)]),
        "schur_solve_host": (I, [P, P, P, I, I, P, ctypes.POINTER(schur_stats)]),
        "schur_complex_solve": (I, [P, P, P, P, I, I, P, ctypes.POINTER(schur_stats)]),
        "schur_apply_mass": (I, [P, P, P, I, I, P]),
        "schur_apply_stiffness": (I, [P, P, P, I, I, P]),
        "schur_apply_S": (I, [P, P, P, I, I, P]),
        "schur_kkt_apply": (I, [P, P, P, I, I, P]),
        "schur_kkt_precond_apply": (I, [P, P, P, I, I, P]),
        "schur_kkt_minres": (I, [P, P, P, I, I, D, I, ctypes.POINTER(I), P]),
        "schur_partition": (I, [ctypes.POINTER(schur_mesh), P, I, ctypes.POINTER(schur_info_t)]),
        "schur_partition_export": (I, [ctypes.POINTER(schur_mesh), P, I, I, P, LL]),
        "schur_get_info": (I, [P, ctypes.POINTER(schur_info_t)]),
        "schur_ndof": (LL, [ctypes.POINTER(schur_mesh)]),
        "schur_destroy": (None, [P]),
        "schur_strerror": (ctypes.c_char_p, [I]),
        "schur_last_error": (ctypes.c_char_p, []),
        "schur_debug_operator": (I, [P, I, I, P, LL]),
        "schur_profile_begin": (I, [ctypes.c_uint]),
        "schur_profile_end": (I, [P, I, ctypes.POINTER(I)]),
        "schur_kernel_category_name": (ctypes.c_char_p, [I]),
        "schur_launch_count": (LL, [P]),
        "schur_apply_S_static": (I, [ctypes.POINTER(schur_mesh), D, P, P, I, I, P]),
        "schur_peak_probe": (I, [I, I, ctypes.POINTER(D), P]),
        "schur_control_solve": (I, [P, P, I, P, P, P, I, I, P, P, ctypes.POINTER(schur_stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code):
    return load().schur_strerror(code).decode()


def last_error():
    return load().schur_last_error().decode()


def _check(code, where, allow=()):
    if code != SCHUR_OK and code not in allow:
        raise SchurError(code, where)
    return code


def schur_profile_begin(mask=0x3FFFF):
    _check(load().schur_profile_begin(mask), "schur_profile_begin")


def schur_profile_end():
    """{category name: (launches, total ms)} since schur_profile_begin (synchronises)."""
    cap = 32  # more than the library's category count
    arr = (schur_kernel_time * cap)()
    cnt = ctypes.c_int(0)
    _check(load().schur_profile_end(arr, cap, ctypes.byref(cnt)), "schur_profile_end")
    return {load().schur_kernel_category_name(arr[k].category).decode(): (arr[k].launches, arr[k].total_ms)
            for k in range(cnt.value)}


PEAK_KINDS = {0: "fp64_fma", 1: "fp32_fma", 2: "fp64_dmma", 3: "tf32_tcgen05"}


def schur_peak_probe(kind, iters, stream=None):
    """Measured TFLOP/s of one arithmetic peak probe (kind: see PEAK_KINDS); synchronises."""
    out = ctypes.c_double(0.0)
    _check(load().schur_peak_probe(int(kind), int(iters), ctypes.byref(out), _stream_ptr(stream)),
           "schur_peak_probe")
    return out.value


def make_mesh(dim, nel):
    nel = [int(nel)] * dim if isinstance(nel, int) else list(nel)
    m = schur_mesh()
    m.dim = dim
    for a in range(dim):
        m.nel[a] = nel[a]
    return m


def default_opts(**kw):
    o = schur_opts()
    load().schur_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "nsub":
            v = [int(v)] * 3 if isinstance(v, int) else list(v) + [1] * (3 - len(v))
            for a in range(3):
                o.nsub[a] = v[a]
        else:
            setattr(o, k, v)
    return o


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


def schur_ndof(dim, nel):
    return int(load().schur_ndof(ctypes.byref(make_mesh(dim, nel))))


def schur_partition(dim, nel, nsub, local_mode=SCHUR_LOCAL_PER_SUBDOMAIN):
    info = schur_info_t()
    ns = (ctypes.c_int * 3)(*([int(nsub)] * 3 if isinstance(nsub, int) else list(nsub) + [1] * (3 - len(nsub))))
    _check(load().schur_partition(ctypes.byref(make_mesh(dim, nel)), ns, local_mode, ctypes.byref(info)),
           "schur_partition")
    return info.as_dict()


def schur_partition_export(dim, nel, nsub, which, local_mode=SCHUR_LOCAL_PER_SUBDOMAIN):
    import numpy as np
    info = schur_partition(dim, nel, nsub, local_mode)
    size = {0: 2 * info["n_lambda"], 1: info["n_delta"], 2: info["n_sub"] * (1 << dim), 3: info["n_sub"]}[which]
    out = np.zeros(max(size, 1), dtype=np.int32)
    ns = (ctypes.c_int * 3)(*([int(nsub)] * 3 if isinstance(nsub, int) else list(nsub) + [1] * (3 - len(nsub))))
    _check(load().schur_partition_export(ctypes.byref(make_mesh(dim, nel)), ns, local_mode, which,
                                         out.ctypes.data_as(ctypes.c_void_p), out.size), "schur_partition_export")
    return out[:size]


class Solver:
    """One schur_ctx: setup at construction, schur_destroy on close()/garbage collection."""

    def __init__(self, dim, nel, beta, nsub=4, precision=SCHUR_FP64, stream=None, **opts):
        self.dim = dim
        self.nel = nel
        self.beta = beta
        self.lib = load()
        self.mesh = make_mesh(dim, nel)
        self.opts = default_opts(nsub=nsub, precision=precision, **opts)
        self.ctx = ctypes.c_void_p()
        _check(self.lib.schur_setup(ctypes.byref(self.mesh), float(beta), ctypes.byref(self.opts),
                                    _stream_ptr(stream), ctypes.byref(self.ctx)), "schur_setup")
        self.n = schur_ndof(dim, nel)
        self.last_stats = None

    def close(self):
        if self.ctx:
            self.lib.schur_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        info = schur_info_t()
        _check(self.lib.schur_get_info(self.ctx, ctypes.byref(info)), "schur_get_info")
        return info.as_dict()

    def _shape(self, t, mult=1):
        if t.dim() == 1:
            return 1, t.numel()
        return t.shape[0], t.shape[1]

    def schur_solve(self, b, x=None, stream=None, allow_notconv=False):
        """x = S^{-1} b; b, x: float64 CUDA tensors of shape (n,) or (nrhs, ld)."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        nrhs, ld = self._shape(b)
        st = schur_stats()
        rc = self.lib.schur_solve(self.ctx, _dptr(b, "b"), _dptr(x, "x"), nrhs, ld, _stream_ptr(stream),
                                  ctypes.byref(st))
        self.last_stats = st.as_dict()
        _check(rc, "schur_solve", allow=(SCHUR_ENOTCONV,) if allow_notconv else ())
        return x

    def schur_solve_host(self, b, x=None, stream=None):
        """Host (numpy float64, C-contiguous) version; copies inside the call."""
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64)
        if x is None:
            x = np.empty_like(b)
        nrhs, ld = (1, b.size) if b.ndim == 1 else b.shape
        st = schur_stats()
        rc = self.lib.schur_solve_host(self.ctx, b.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p),
                                       nrhs, ld, _stream_ptr(stream), ctypes.byref(st))
        self.last_stats = st.as_dict()
        _check(rc, "schur_solve_host")
        return x

    def schur_complex_solve(self, bre, bim=None, stream=None):
        """z = (K + i gamma M)^{-1} (bre + i bim) as a complex128 CUDA tensor."""
        import torch
        nrhs, ld = self._shape(bre)
        z = torch.empty((nrhs, ld, 2), dtype=torch.float64, device=bre.device)
        st = schur_stats()
        rc = self.lib.schur_complex_solve(self.ctx, _dptr(bre, "bre"), None if bim is None else _dptr(bim, "bim"),
                                          ctypes.c_void_p(z.data_ptr()), nrhs, ld, _stream_ptr(stream), ctypes.byref(st))
        self.last_stats = st.as_dict()
        _check(rc, "schur_complex_solve")
        zc = torch.view_as_complex(z)
        return zc[0] if bre.dim() == 1 else zc

    def _apply(self, fn, x, y, stream, where):
        import torch
        if y is None:
            y = torch.empty_like(x)
        nrhs, ld = self._shape(x)
        _check(fn(self.ctx, _dptr(x, "x"), _dptr(y, "y"), nrhs, ld, _stream_ptr(stream)), where)
        return y

    def schur_apply_mass(self, x, y=None, stream=None):
        return self._apply(self.lib.schur_apply_mass, x, y, stream, "schur_apply_mass")

    def schur_apply_stiffness(self, x, y=None, stream=None):
        return self._apply(self.lib.schur_apply_stiffness, x, y, stream, "schur_apply_stiffness")

    def schur_apply_S(self, x, y=None, stream=None):
        return self._apply(self.lib.schur_apply_S, x, y, stream, "schur_apply_S")

    def schur_control_solve(self, ybar_full, stream=None, want_violation=True):
        """Range-space solve with Dirichlet data: ybar_full (float64 CUDA tensor, (nfull,) or
        (nrhs, nfull) over all grid nodes) -> (y, u, lambda, violation per column or None)."""
        import numpy as np
        import torch
        nrhs, ldf = self._shape(ybar_full)
        shape = (self.n,) if ybar_full.dim() == 1 else (nrhs, self.n)
        y = torch.empty(shape, dtype=torch.float64, device=ybar_full.device)
        u = torch.empty_like(y)
        lam = torch.empty_like(y)
        viol = np.zeros(max(nrhs, 1)) if want_violation else None
        st = schur_stats()
        rc = self.lib.schur_control_solve(self.ctx, _dptr(ybar_full, "ybar_full"), ldf, _dptr(y, "y"), _dptr(u, "u"),
                                          _dptr(lam, "lambda"), nrhs, self.n,
                                          None if viol is None else viol.ctypes.data_as(ctypes.c_void_p),
                                          _stream_ptr(stream), ctypes.byref(st))
        self.last_stats = st.as_dict()
        _check(rc, "schur_control_solve")
        return y, u, lam, (None if viol is None else viol[:nrhs])

    def schur_kkt_apply(self, v, r=None, stream=None):
        return self._apply(self.lib.schur_kkt_apply, v, r, stream, "schur_kkt_apply")

    def schur_kkt_precond_apply(self, r, z=None, stream=None):
        return self._apply(self.lib.schur_kkt_precond_apply, r, z, stream, "schur_kkt_precond_apply")

    def schur_kkt_minres(self, rhs, sol=None, tol=1e-10, max_it=50, stream=None):
        import torch
        if sol is None:
            sol = torch.zeros_like(rhs)
        nrhs, ld = self._shape(rhs)
        it = ctypes.c_int(0)
        _check(self.lib.schur_kkt_minres(self.ctx, _dptr(rhs, "rhs"), _dptr(sol, "sol"), nrhs, ld, float(tol),
                                         int(max_it), ctypes.byref(it), _stream_ptr(stream)), "schur_kkt_minres")
        return sol, it.value

    def schur_debug_operator(self, which, cls=0):
        import numpy as np
        info = self.info()
        nD, nc, nco = info["n_delta"], 1 << self.dim, info["n_coarse"]
        s1 = [self.nel // n for n in (self.opts.nsub[a] for a in range(self.dim))][0] + 1
        shape = {0: (nD, nD), 1: (nD, nc), 2: (nD, nD), 3: (nco, nco), 4: (nco, nco),
                 6: (s1, s1 ** (self.dim - 1), s1 ** (self.dim - 1))}[which]
        out = np.zeros(shape + (2,), dtype=np.float64)
        _check(self.lib.schur_debug_operator(self.ctx, which, cls, out.ctypes.data_as(ctypes.c_void_p),
                                             out.size // 2), "schur_debug_operator")
        return out[..., 0] + 1j * out[..., 1]


class schur_server_opts(ctypes.Structure):
    _fields_ = [("device_mem_budget", ctypes.c_size_t), ("workers", ctypes.c_int), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_batch_rhs", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class schur_server_info_t(ctypes.Structure):
    _fields_ = [("cached_contexts", ctypes.c_int), ("queued", ctypes.c_int), ("completed", ctypes.c_longlong),
                ("bytes_reserved", ctypes.c_longlong), ("batches", ctypes.c_longlong),
                ("batch_columns", ctypes.c_longlong), ("shared_requests", ctypes.c_longlong),
                ("setups", ctypes.c_longlong), ("max_concurrent", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


def _load_server_syms(lib):
    if getattr(lib, "_server_bound", False):
        return lib
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.schur_server_default_opts.restype = None
    lib.schur_server_default_opts.argtypes = [ctypes.POINTER(schur_server_opts)]
    lib.schur_server_create.restype = I
    lib.schur_server_create.argtypes = [ctypes.POINTER(schur_server_opts), ctypes.POINTER(P)]
    lib.schur_submit.restype = I
    lib.schur_submit.argtypes = [P, ctypes.POINTER(schur_mesh), D, P, I, P, ctypes.POINTER(LL)]
    lib.schur_poll.restype = I
    lib.schur_poll.argtypes = [P, LL, ctypes.POINTER(schur_stats)]
    lib.schur_wait.restype = I
    lib.schur_wait.argtypes = [P, LL, D, ctypes.POINTER(schur_stats)]
    lib.schur_server_info.restype = I
    lib.schur_server_info.argtypes = [P, ctypes.POINTER(schur_server_info_t)]
    lib.schur_server_destroy.restype = None
    lib.schur_server_destroy.argtypes = [P]
    lib._server_bound = True
    return lib


class Server:
    """schur_server: submit host right-hand sides, poll or wait for host results."""

    def __init__(self, budget_bytes=16 << 30, workers=4, precision=SCHUR_MIXED, tol=1e-10, max_batch_rhs=16,
                 max_iter=300):
        self.lib = _load_server_syms(load())
        o = schur_server_opts()
        self.lib.schur_server_default_opts(ctypes.byref(o))
        o.device_mem_budget = int(budget_bytes)
        o.workers = workers
        o.precision = precision
        o.tol = tol
        o.max_batch_rhs = max_batch_rhs
        o.max_iter = max_iter
        self.srv = ctypes.c_void_p()
        _check(self.lib.schur_server_create(ctypes.byref(o), ctypes.byref(self.srv)), "schur_server_create")
        self._bufs = {}
        _live_servers.add(self)

    def submit(self, dim, nel, beta, b):
        """b: float64 host array (n,) or (nrhs, n); returns a ticket."""
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        t = ctypes.c_longlong(0)
        rc = self.lib.schur_submit(self.srv, ctypes.byref(make_mesh(dim, nel)), float(beta),
                                   b.ctypes.data_as(ctypes.c_void_p), nrhs, x.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(t))
        _check(rc, "schur_submit")
        self._bufs[t.value] = (b, x)
        return t.value

    def poll(self, ticket):
        """(done, x or None, stats)"""
        st = schur_stats()
        rc = self.lib.schur_poll(self.srv, ticket, ctypes.byref(st))
        if rc == 1:
            return False, None, None
        _check(rc, "schur_poll")
        return True, self._bufs.pop(ticket)[1], st.as_dict()

    def wait(self, ticket, timeout_ms=600000.0):
        st = schur_stats()
        _check(self.lib.schur_wait(self.srv, ticket, float(timeout_ms), ctypes.byref(st)), "schur_wait")
        return self._bufs.pop(ticket)[1], st.as_dict()

    def info(self):
        i = schur_server_info_t()
        _check(self.lib.schur_server_info(self.srv, ctypes.byref(i)), "schur_server_info")
        return {k: getattr(i, k) for k, _ in i._fields_ if k != "reserved"}

    def close(self):
        if self.srv:
            self.lib.schur_server_destroy(self.srv)
            self.srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Servers own worker threads that call CUDA; close any still open before the interpreter (and then
# the CUDA runtime) shuts down.
import atexit as _atexit
import weakref as _weakref

_live_servers = _weakref.WeakSet()


@_atexit.register
def _close_live_servers():
    for s in list(_live_servers):
        try:
            s.close()
        except Exception:
            pass
