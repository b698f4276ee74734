"""Thin Python binding of libqn (include/qn.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels. PyTorch supplies device memory and the current CUDA stream.
The functions carry the C-ABI names; a missing library is a hard error.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqn.so")

QN_OK = 0
QN_EINVAL = -1
QN_ENOMEM = -2
QN_ECUDA = -3
QN_ENOTCONV = -4
QN_EDIVERGED = -5
QN_ETIMEOUT = -6
QN_EUNSUPPORTED = -7

QN_BC_DIRICHLET = 0
QN_BC_NEUMANN = 1
QN_BC_ROBIN = 2
BCS = {"dirichlet": QN_BC_DIRICHLET, "neumann": QN_BC_NEUMANN, "robin": QN_BC_ROBIN}
QN_PREC_FP64 = 0
QN_PREC_BF16X3 = 1
QN_PREC_BF16X6 = 2
QN_BETA_PAPER = 0
QN_BETA_FIXED = 1

PRECISIONS = {"fp64": QN_PREC_FP64, "bf16x3": QN_PREC_BF16X3, "bf16x6": QN_PREC_BF16X6}


class QnProblem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("bc", ctypes.c_int),
                ("precision", ctypes.c_int), ("lam", ctypes.c_double), ("b", ctypes.c_double),
                ("length", ctypes.c_double), ("potential_host", ctypes.POINTER(ctypes.c_double)),
                ("sem_k", ctypes.c_int), ("robin_kappa", ctypes.c_double)]


class QnStats(ctypes.Structure):
    _fields_ = [("res_norm", ctypes.c_double), ("f_norm", ctypes.c_double),
                ("fu_min", ctypes.c_double), ("fu_max", ctypes.c_double),
                ("beta", ctypes.c_double), ("rel", ctypes.c_double), ("lambda", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class QnOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_it", ctypes.c_int), ("beta_mode", ctypes.c_int),
                ("beta_value", ctypes.c_double), ("step", ctypes.c_double),
                ("sync_every", ctypes.c_int), ("graph", ctypes.c_int)]


class QnResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel", ctypes.c_double)]


class QnProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong),
                ("residual_launches", ctypes.c_int), ("residual_ms", ctypes.c_double),
                ("finalize_launches", ctypes.c_int), ("finalize_ms", ctypes.c_double),
                ("modeprod_launches", ctypes.c_int), ("modeprod_ms", ctypes.c_double),
                ("mp_store_launches", ctypes.c_int), ("mp_store_ms", ctypes.c_double),
                ("mp_divide_launches", ctypes.c_int), ("mp_divide_ms", ctypes.c_double),
                ("mp_last_launches", ctypes.c_int), ("mp_last_ms", ctypes.c_double),
                ("residual_tiled_launches", ctypes.c_int), ("residual_tiled_ms", ctypes.c_double),
                ("split_products", ctypes.c_int), ("x6_from", ctypes.c_int),
                ("fused_launches", ctypes.c_int), ("fused_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class QnSysInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("alpha", ctypes.c_double), ("D", ctypes.c_double),
                ("U", ctypes.c_void_p), ("V", ctypes.c_void_p), ("f1", ctypes.c_void_p),
                ("f2", ctypes.c_void_p)]


class QnSysResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel", ctypes.c_double),
                ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class QnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqn error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqn.so (built by paper_2502_03611_gb300.build). No fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libqn.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    sig = {
        "qn_version": (ctypes.c_int, []),
        "qn_last_error": (ctypes.c_char_p, []),
        "qn_setup_1d_eig": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, D, D, D]),
        "qn_setup_1d_robin": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D, D]),
        "qn_setup_1d_sem": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, D, D, D, D, D]),
        "qn_ctx_create": (ctypes.c_int, [ctypes.POINTER(QnProblem), ctypes.POINTER(P)]),
        "qn_ctx_destroy": (ctypes.c_int, [P]),
        "qn_residual": (ctypes.c_int, [P, P, P, P, ctypes.POINTER(QnStats), P]),
        "qn_fast_diag_solve": (ctypes.c_int, [P, P, P, ctypes.c_double, P]),
        "qn_step": (ctypes.c_int, [P, P, P, ctypes.c_double, ctypes.POINTER(QnStats), P]),
        "qn_solve": (ctypes.c_int, [P, P, P, ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult),
                                    ctypes.POINTER(QnStats), ctypes.c_int, P]),
        "qn_solve_host_zero_start": (ctypes.c_int, [P, P, P, ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult),
                                                    ctypes.POINTER(QnStats), ctypes.c_int, P]),
        "qn_solve_host": (ctypes.c_int, [P, P, P, ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult),
                                         ctypes.POINTER(QnStats), ctypes.c_int, P]),
        "qn_solve_host_many": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int,
                                              ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult), P]),
        "qn_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "qn_test_withhold_arrival": (ctypes.c_int, []),
        "qn_residual_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               P, P, P, ctypes.POINTER(QnStats), P]),
        "qn_batch_create": (ctypes.c_int, [ctypes.POINTER(QnSysInstance), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(P)]),
        "qn_batch_solve": (ctypes.c_int, [P, ctypes.POINTER(QnOpts), ctypes.POINTER(QnSysResult), P]),
        "qn_batch_destroy": (ctypes.c_int, [P]),
        "qn_autotune_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "qn_net_param_count": (ctypes.c_longlong, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "qn_net_create": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.POINTER(P)]),
        "qn_net_destroy": (ctypes.c_int, [P]),
        "qn_net_set_params": (ctypes.c_int, [P, P, ctypes.c_longlong]),
        "qn_net_get_params": (ctypes.c_int, [P, P, ctypes.c_longlong]),
        "qn_net_forward": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
        "qn_net_gradients": (ctypes.c_int, [P, P, P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_double), P]),
        "qn_net_train_step": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                             ctypes.POINTER(ctypes.c_double), P]),
        "qn_net_predict": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]),
        "qn_interp3d": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]),
        "qn_interp3d_f32": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]),
        "qn_solve_warm": (ctypes.c_int, [P, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult),
                                         ctypes.POINTER(ctypes.c_int), P]),
        "qn_profile_read": (ctypes.c_int, [P, ctypes.POINTER(QnProfile)]),
        "qn_set_escalation": (ctypes.c_int, [P, ctypes.c_double]),
        "qn_set_fused_residual": (ctypes.c_int, [P, ctypes.c_int]),
        "qn_eig_solve": (ctypes.c_int, [P, P, ctypes.POINTER(QnOpts), ctypes.POINTER(QnResult),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(QnStats), ctypes.c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, allowed=(QN_OK,)):
    if rc not in allowed:
        raise QnError(rc, load_library().qn_last_error().decode())
    return rc


def qn_version() -> int:
    return load_library().qn_version()


def qn_last_error() -> str:
    return load_library().qn_last_error().decode()


def qn_setup_1d_eig(n: int, h: float | None = None, bc: int = QN_BC_DIRICHLET):
    """Host 1-D diagonalisation; returns numpy (S, S_inv, lam)."""
    lib = load_library()
    h = 1.0 / (n + 1) if h is None else h
    S = np.empty((n, n))
    Si = np.empty((n, n))
    lam = np.empty(n)
    D = ctypes.POINTER(ctypes.c_double)
    _check(lib.qn_setup_1d_eig(n, h, bc, S.ctypes.data_as(D), Si.ctypes.data_as(D), lam.ctypes.data_as(D)))
    return S, Si, lam


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, numel, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


class QnContext:
    """Owns a qn_ctx (qn_ctx_create / qn_ctx_destroy)."""

    def __init__(self, dim: int, n: int, precision: str | int = "fp64", lam: float = 0.0,
                 b: float = 1.0, bc: str | int = QN_BC_DIRICHLET, length: float = 0.0, potential=None,
                 sem_k: int = 0, robin_kappa: float = 0.0):
        """potential: None, or the 1-D tables of V = v_x + v_y (+ v_z) at the nodes, an array
        of shape (n,) (the same table on every axis) or (dim, n) (x first)."""
        lib = load_library()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        bcv = BCS[bc] if isinstance(bc, str) else int(bc)
        pot = None
        if potential is not None:
            v = np.asarray(potential, dtype=np.float64)
            pot = np.ascontiguousarray(np.broadcast_to(v, (dim, n)) if v.ndim == 1 else v)
            if pot.shape != (dim, n):
                raise ValueError(f"potential tables must have shape ({n},) or ({dim}, {n})")
        ptr = pot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if pot is not None else None
        self.problem = QnProblem(dim, n, bcv, prec, lam, b, length, ptr, sem_k, robin_kappa)
        self.dim, self.n, self.precision, self.bc = dim, n, prec, bcv
        self.numel = n ** dim
        h = ctypes.c_void_p()
        _check(lib.qn_ctx_create(ctypes.byref(self.problem), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().qn_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def qn_ctx_create(dim, n, precision="fp64", lam=0.0, b=1.0, bc=QN_BC_DIRICHLET, length=0.0,
                  potential=None, sem_k=0) -> QnContext:
    return QnContext(dim, n, precision, lam, b, bc, length, potential, sem_k)


def qn_setup_1d_robin(n: int, h: float, kappa: float):
    """Host Robin diagonalisation; returns numpy (S, S_inv, lam)."""
    lib = load_library()
    S = np.empty((n, n))
    Si = np.empty((n, n))
    lam = np.empty(n)
    D = ctypes.POINTER(ctypes.c_double)
    _check(lib.qn_setup_1d_robin(n, h, kappa, S.ctypes.data_as(D), Si.ctypes.data_as(D), lam.ctypes.data_as(D)))
    return S, Si, lam


def qn_setup_1d_sem(n: int, k: int, length: float = 1.0, bc: int = QN_BC_DIRICHLET):
    """Host Q^k spectral element matrices; returns numpy (H, S, S_inv, lam, nodes)."""
    lib = load_library()
    H = np.empty((n, n))
    S = np.empty((n, n))
    Si = np.empty((n, n))
    lam = np.empty(n)
    x = np.empty(n)
    D = ctypes.POINTER(ctypes.c_double)
    _check(lib.qn_setup_1d_sem(n, k, length, bc, H.ctypes.data_as(D), S.ctypes.data_as(D), Si.ctypes.data_as(D),
                               lam.ctypes.data_as(D), x.ctypes.data_as(D)))
    return H, S, Si, lam, x


def qn_ctx_destroy(ctx: QnContext):
    ctx.close()


def qn_residual(ctx: QnContext, U, f, R=None, stream=None) -> dict:
    st = QnStats()
    _check(load_library().qn_residual(ctx.handle, _dptr(U, ctx.numel, "U"), _dptr(f, ctx.numel, "f"),
                                      _dptr(R, ctx.numel, "R"), ctypes.byref(st), _stream_ptr(stream)))
    return st.as_dict()


def qn_fast_diag_solve(ctx: QnContext, r, V, shift: float, stream=None):
    _check(load_library().qn_fast_diag_solve(ctx.handle, _dptr(r, ctx.numel, "r"), _dptr(V, ctx.numel, "V"),
                                             float(shift), _stream_ptr(stream)))


def qn_step(ctx: QnContext, U, f, beta: float = math.nan, stream=None) -> dict:
    st = QnStats()
    _check(load_library().qn_step(ctx.handle, _dptr(U, ctx.numel, "U"), _dptr(f, ctx.numel, "f"),
                                  float(beta), ctypes.byref(st), _stream_ptr(stream)))
    return st.as_dict()


def make_opts(tol=1e-10, max_it=200, beta=None, step=1.0, sync_every=2, graph=False) -> QnOpts:
    if beta is None:
        return QnOpts(tol, max_it, QN_BETA_PAPER, 0.0, step, sync_every, 1 if graph else 0)
    return QnOpts(tol, max_it, QN_BETA_FIXED, float(beta), step, sync_every, 1 if graph else 0)


def qn_solve(ctx: QnContext, U, f, tol=1e-10, max_it=200, beta=None, step=1.0, sync_every=2,
             history_len=0, stream=None, check=True, graph=False):
    """Returns (result dict, list of per-iterate stats dicts)."""
    opts = make_opts(tol, max_it, beta, step, sync_every, graph)
    res = QnResult()
    hist = (QnStats * history_len)() if history_len > 0 else None
    rc = load_library().qn_solve(ctx.handle, _dptr(U, ctx.numel, "U"), _dptr(f, ctx.numel, "f"),
                                 ctypes.byref(opts), ctypes.byref(res), hist, history_len,
                                 _stream_ptr(stream))
    if check:
        _check(rc, allowed=(QN_OK, QN_ENOTCONV, QN_EDIVERGED))
    out = {"iterations": res.iterations, "status": res.status, "rel": res.rel, "rc": rc}
    n_h = min(res.iterations + 1, history_len) if rc in (QN_OK, QN_ENOTCONV, QN_EDIVERGED) else 0
    return out, [hist[i].as_dict() for i in range(n_h)] if hist is not None else []


def qn_eig_solve(ctx: QnContext, U, tol=1e-10, max_it=4096, beta=None, step=1.0, sync_every=8,
                 history_len=0, stream=None, graph=False):
    """Nonlinear eigenproblem; U (device) holds the start and receives the normalised
    eigenfunction. Returns (result dict with "lambda", list of per-iterate stats dicts)."""
    opts = make_opts(tol, max_it, beta, step, sync_every, graph)
    res = QnResult()
    lam = ctypes.c_double()
    hist = (QnStats * history_len)() if history_len > 0 else None
    rc = load_library().qn_eig_solve(ctx.handle, _dptr(U, ctx.numel, "U"), ctypes.byref(opts), ctypes.byref(res),
                                     ctypes.byref(lam), hist, history_len, _stream_ptr(stream))
    _check(rc, allowed=(QN_OK, QN_ENOTCONV, QN_EDIVERGED))
    out = {"iterations": res.iterations, "status": res.status, "rel": res.rel, "lambda": lam.value, "rc": rc}
    n_h = min(res.iterations + 1, history_len)
    return out, [hist[i].as_dict() for i in range(n_h)] if hist is not None else []


def qn_solve_host(ctx: QnContext, U_host: np.ndarray, f_host: np.ndarray, tol=1e-10, max_it=200,
                  beta=None, step=1.0, sync_every=2, stream=None, graph=False, zero_start=False):
    """Solve with host arrays (copies inside the call). U_host is updated in place; with
    zero_start the solve starts from U = 0 and U_host is output only (qn_solve_host_zero_start:
    no copy of a start)."""
    for name, a in (("U_host", U_host), ("f_host", f_host)):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != ctx.numel:
            raise ValueError(f"{name} must be a C-contiguous float64 array of {ctx.numel} values")
    opts = make_opts(tol, max_it, beta, step, sync_every, graph)
    res = QnResult()
    lib = load_library()
    fn = lib.qn_solve_host_zero_start if zero_start else lib.qn_solve_host
    rc = fn(ctx.handle, ctypes.c_void_p(U_host.ctypes.data), ctypes.c_void_p(f_host.ctypes.data),
            ctypes.byref(opts), ctypes.byref(res), None, 0, _stream_ptr(stream))
    _check(rc, allowed=(QN_OK, QN_ENOTCONV, QN_EDIVERGED))
    return {"iterations": res.iterations, "status": res.status, "rel": res.rel, "rc": rc}


def qn_solve_host_many(ctx: QnContext, U_hosts, f_hosts, tol=1e-10, max_it=200, beta=None, step=1.0,
                       sync_every=2, stream=None, graph=False, zero_start=False):
    """A sequence of host-array solves, copies overlapped with the neighbouring solves
    (qn_solve_host_many). U_hosts[i], f_hosts[i]: C-contiguous float64 numpy arrays (the
    same array may appear more than once, see the header). Returns one result dict per
    problem."""
    if len(U_hosts) != len(f_hosts):
        raise ValueError("U_hosts and f_hosts must have the same length")
    for name, arrs in (("U_hosts", U_hosts), ("f_hosts", f_hosts)):
        for a in arrs:
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != ctx.numel:
                raise ValueError(f"{name} entries must be C-contiguous float64 arrays of {ctx.numel} values")
    count = len(U_hosts)
    Up = (ctypes.c_void_p * max(count, 1))(*[a.ctypes.data for a in U_hosts])
    fp = (ctypes.c_void_p * max(count, 1))(*[a.ctypes.data for a in f_hosts])
    res = (QnResult * max(count, 1))()
    opts = make_opts(tol, max_it, beta, step, sync_every, graph)
    _check(load_library().qn_solve_host_many(ctx.handle, count, Up, fp, 1 if zero_start else 0, ctypes.byref(opts),
                                             res, _stream_ptr(stream)))
    return [{"iterations": res[i].iterations, "status": res[i].status, "rel": res[i].rel} for i in range(count)]


def qn_test_withhold_arrival():
    """Test-only: the next tensor-core mode-product launch withholds one TMA arrival and its
    waits give up after 2 s with QN_ETIMEOUT (bounded; no GPU fault)."""
    _check(load_library().qn_test_withhold_arrival())


def qn_set_escalation(ctx: QnContext, rate: float):
    """BF16X3 solves switch their backward products to the six-product level when the
    observed contraction exceeds `rate` and twice the quasi-Newton bound (0: off)."""
    _check(load_library().qn_set_escalation(ctx.handle, float(rate)))


def qn_set_fused_residual(ctx: QnContext, on: bool = True):
    """Iterations >= 1 of the 3-D split solve evaluate the residual inside the first
    forward mode product (one kernel) instead of the separate residual kernel."""
    _check(load_library().qn_set_fused_residual(ctx.handle, 1 if on else 0))


def qn_profile_enable(ctx: QnContext, on: bool = True):
    _check(load_library().qn_profile_enable(ctx.handle, 1 if on else 0))


def qn_profile_read(ctx: QnContext) -> dict:
    p = QnProfile()
    _check(load_library().qn_profile_read(ctx.handle, ctypes.byref(p)))
    return p.as_dict()


def qn_autotune_tile(n: int, copies: int = 16):
    """Project autotuner: fastest (bk, bn) for the grouped mode product at size n."""
    bk, bn, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load_library().qn_autotune_tile(n, copies, ctypes.byref(bk), ctypes.byref(bn), ctypes.byref(ms)))
    return bk.value, bn.value, ms.value


class QnBatch:
    """Owns a qn_batch over coupled 2-D instances. `instances` is a list of
    dicts with n, alpha, D and float64 CUDA tensors U, V, f1, f2 (n*n each);
    the tensors must outlive the batch (the object keeps references)."""

    def __init__(self, instances, bk: int = 0, bn=None):
        lib = load_library()
        self._keep = instances
        arr = (QnSysInstance * len(instances))()
        for i, d in enumerate(instances):
            nn = d["n"] * d["n"]
            arr[i] = QnSysInstance(d["n"], d["alpha"], d["D"], _dptr(d["U"], nn, "U"), _dptr(d["V"], nn, "V"),
                                   _dptr(d["f1"], nn, "f1"), _dptr(d["f2"], nn, "f2"))
        bnarr = None
        if bn is not None:
            bnarr = (ctypes.c_int * len(instances))(*[int(x) for x in bn])
        h = ctypes.c_void_p()
        _check(lib.qn_batch_create(arr, len(instances), int(bk), bnarr, ctypes.byref(h)))
        self._h = h
        self.count = len(instances)

    def solve(self, tol=1e-10, max_it=200, sync_every=4, stream=None):
        opts = make_opts(tol, max_it, None, 1.0, sync_every)
        res = (QnSysResult * self.count)()
        rc = load_library().qn_batch_solve(self._h, ctypes.byref(opts), res, _stream_ptr(stream))
        _check(rc, allowed=(QN_OK, QN_ENOTCONV, QN_EDIVERGED))
        return rc, [r.as_dict() for r in res]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().qn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fptr(t, numel, name, dtype="float32"):
    import torch
    want = torch.float32 if dtype == "float32" else torch.float64
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def qn_interp3d(src, m_from: int, dst, m_to: int, batch: int = 1, scale: float = 1.0, stream=None):
    """Trilinear transfer of `batch` fields between interior grids (device tensors)."""
    lib = load_library()
    if dst.dtype.is_floating_point and dst.element_size() == 4:
        _check(lib.qn_interp3d_f32(_fptr(src, batch * m_from ** 3, "src", "float64"), m_from,
                                   _fptr(dst, batch * m_to ** 3, "dst", "float32"), m_to, batch, scale,
                                   _stream_ptr(stream)))
    else:
        _check(lib.qn_interp3d(_fptr(src, batch * m_from ** 3, "src", "float64"), m_from,
                               _fptr(dst, batch * m_to ** 3, "dst", "float64"), m_to, batch, scale,
                               _stream_ptr(stream)))


class QnNet:
    """Owns a qn_net (learned warm start)."""

    def __init__(self, G: int, modes: int = 6, blocks: int = 4, max_batch: int = 8, channels: int = 32):
        lib = load_library()
        self.G, self.M, self.L, self.C, self.max_batch = G, modes, blocks, channels, max_batch
        self.nparams = lib.qn_net_param_count(channels, modes, blocks)
        h = ctypes.c_void_p()
        _check(lib.qn_net_create(G, channels, modes, blocks, max_batch, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load_library().qn_net_set_params(self._h, ctypes.c_void_p(p.ctypes.data), p.size))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparams, dtype=np.float32)
        _check(load_library().qn_net_get_params(self._h, ctypes.c_void_p(p.ctypes.data), p.size))
        return p

    def forward(self, f_coarse, out, batch: int, stream=None):
        n = batch * self.G ** 3
        _check(load_library().qn_net_forward(self._h, _fptr(f_coarse, n, "f"), _fptr(out, n, "out"), batch,
                                             _stream_ptr(stream)))

    def gradients(self, f_coarse, target, batch: int, grads, stream=None) -> float:
        n = batch * self.G ** 3
        loss = ctypes.c_double()
        _check(load_library().qn_net_gradients(self._h, _fptr(f_coarse, n, "f"), _fptr(target, n, "target"), batch,
                                               _fptr(grads, self.nparams, "grads"), ctypes.byref(loss),
                                               _stream_ptr(stream)))
        return loss.value

    def train_step(self, f_coarse, target, batch: int, lr: float, weight_decay: float = 0.0, stream=None,
                   want_loss: bool = True):
        n = batch * self.G ** 3
        loss = ctypes.c_double()
        _check(load_library().qn_net_train_step(self._h, _fptr(f_coarse, n, "f"), _fptr(target, n, "target"), batch,
                                                ctypes.c_float(lr), ctypes.c_float(weight_decay),
                                                ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)))
        return loss.value if want_loss else None

    def predict(self, f_fine, n: int, U0, in_scale: float = 1.0, out_scale: float = 1.0, stream=None):
        _check(load_library().qn_net_predict(self._h, _fptr(f_fine, n ** 3, "f", "float64"), n, in_scale, out_scale,
                                             _fptr(U0, n ** 3, "U0", "float64"), _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().qn_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qn_solve_warm(ctx: QnContext, net: QnNet, U, f, in_scale=1.0, out_scale=1.0, tol=1e-10, max_it=200,
                  sync_every=2, stream=None):
    opts = make_opts(tol, max_it, None, 1.0, sync_every)
    res = QnResult()
    used = ctypes.c_int()
    rc = load_library().qn_solve_warm(ctx.handle, net.handle, _dptr(U, ctx.numel, "U"), _dptr(f, ctx.numel, "f"),
                                      ctx.n, in_scale, out_scale, ctypes.byref(opts), ctypes.byref(res),
                                      ctypes.byref(used), _stream_ptr(stream))
    _check(rc, allowed=(QN_OK, QN_ENOTCONV, QN_EDIVERGED))
    return {"iterations": res.iterations, "status": res.status, "rel": res.rel, "used_warm": bool(used.value)}
