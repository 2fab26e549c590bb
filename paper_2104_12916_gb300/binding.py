"""ctypes binding of libpcgipm.so: the C ABI of include/pcgipm.h with the same names.

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays are either host numpy float64 arrays (C-contiguous) or torch CUDA
float64 tensors (contiguous); the pointer kind is taken from the arrays.
Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

QP_OK, QP_EINVAL, QP_ENOMEM, QP_ESINGULAR, QP_ENOTCONVEX = 0, -1, -2, -3, -4
QP_EMAXIT, QP_ENUMERIC, QP_ETIMEOUT, QP_EAGAIN, QP_ECUDA, QP_ESTATE = -5, -6, -7, -8, -9, -10
QP_PREC_FP64, QP_PREC_FP32 = 0, 1
QP_PC_AUTO, QP_PC_PL, QP_PC_PH_EXACT, QP_PC_PH_DIAG, QP_PC_NONE = 0, 1, 2, 3, 4
QP_MODE_PARITY, QP_MODE_PAPER = 0, 1
QP_FORM_AUTO = -1
QP_PTR_HOST, QP_PTR_DEVICE = 0, 1

EXPORTED = [
    "qp_opts_default", "qp_create", "qp_factor_K0", "qp_kf_apply", "qp_k0_solve",
    "qp_pcg_reduced_solve", "qp_ipm_solve", "qp_get_stats", "qp_device_bytes",
    "qp_pcg_bytes_per_iter", "qp_time_pcg_iteration", "qp_kernel_launches", "qp_destroy", "qp_strerror",
    "qp_kf_apply_static", "qp_batch_solve", "qp_get_solution", "qp_create_csr", "qp_device_bytes_bound",
    "qp_server_create", "qp_server_submit", "qp_server_poll", "qp_server_drain", "qp_server_get_stats",
    "qp_server_destroy",
]


class qp_opts(ct.Structure):
    _fields_ = [
        ("precision", ct.c_int), ("precond", ct.c_int), ("pcg_mode", ct.c_int),
        ("max_ipm", ct.c_int), ("max_pcg", ct.c_int), ("refine_max", ct.c_int),
        ("pcg_tol", ct.c_double), ("refine_tol", ct.c_double), ("tol_feas", ct.c_double),
        ("tol_mu", ct.c_double), ("pcg_check_every", ct.c_int), ("mixed_fallback", ct.c_int),
        ("pcg_blocks", ct.c_int), ("blocking_wait", ct.c_int), ("pcg_form", ct.c_int),
        ("factor_tc", ct.c_int), ("autotune", ct.c_int), ("factor_bk", ct.c_int), ("stream", ct.c_void_p),
    ]


class qp_result(ct.Structure):
    _fields_ = [
        ("status", ct.c_int), ("ipm_iters", ct.c_int), ("pcg_iters", ct.c_longlong),
        ("obj", ct.c_double), ("res_p", ct.c_double), ("res_d", ct.c_double), ("mu", ct.c_double),
        ("solve_ms", ct.c_double), ("wait_ms", ct.c_double), ("latency_ms", ct.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qp_problem(ct.Structure):
    _fields_ = [
        ("n", ct.c_int), ("m1", ct.c_int), ("m2", ct.c_int),
        ("H", ct.c_void_p), ("c", ct.c_void_p), ("A", ct.c_void_p), ("b", ct.c_void_p),
        ("C", ct.c_void_p), ("C_rowptr", ct.c_void_p), ("C_colidx", ct.c_void_p), ("C_val", ct.c_void_p),
        ("d", ct.c_void_p),
    ]


class qp_server_stats(ct.Structure):
    _fields_ = [
        ("submitted", ct.c_longlong), ("completed", ct.c_longlong), ("failed", ct.c_longlong),
        ("queued", ct.c_int), ("active", ct.c_int), ("reserved_bytes", ct.c_size_t),
        ("peak_reserved_bytes", ct.c_size_t), ("peak_device_bytes", ct.c_size_t),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qp_stats(ct.Structure):
    _fields_ = [
        ("status", ct.c_int), ("precond_used", ct.c_int), ("ipm_iters", ct.c_int),
        ("pcg_iters_total", ct.c_longlong), ("newton_solves", ct.c_int), ("refine_sweeps", ct.c_int),
        ("res_p", ct.c_double), ("res_d", ct.c_double), ("mu", ct.c_double), ("obj", ct.c_double),
        ("t_factor_ms", ct.c_double), ("t_solve_ms", ct.c_double), ("t_pcg_ms", ct.c_double),
        ("t_precond_ms", ct.c_double), ("op64_solves", ct.c_int), ("op64_switch_iter", ct.c_int),
        ("pc64_switch_iter", ct.c_int),
        ("pc_switch_iter", ct.c_int), ("factor_tc", ct.c_int), ("pcg_form_used", ct.c_int),
        ("pcg_grid", ct.c_int), ("k0_inertia_pos", ct.c_int), ("k0_inertia_neg", ct.c_int),
        ("k0_pivots_2x2", ct.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libpcgipm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libpcgipm.so not built at {path}: run paper_2104_12916_gb300.build.build()")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    D = ct.c_double
    I = ct.c_int
    lib.qp_opts_default.argtypes = [ct.POINTER(qp_opts)]
    lib.qp_opts_default.restype = None
    lib.qp_create.argtypes = [ct.POINTER(P), I, I, I, P, P, P, P, P, P, ct.POINTER(qp_opts), I]
    lib.qp_create_csr.argtypes = [ct.POINTER(P), I, I, I, P, P, P, P, P, P, P, P, ct.POINTER(qp_opts), I]
    lib.qp_create_csr.restype = I
    lib.qp_device_bytes_bound.argtypes = [I, I, I, ct.POINTER(qp_opts)]
    lib.qp_device_bytes_bound.restype = ct.c_size_t
    lib.qp_server_create.argtypes = [ct.POINTER(P), ct.c_size_t, I, ct.POINTER(qp_opts)]
    lib.qp_server_create.restype = I
    lib.qp_server_submit.argtypes = [P, ct.POINTER(qp_problem), ct.POINTER(ct.c_ulonglong)]
    lib.qp_server_submit.restype = I
    lib.qp_server_poll.argtypes = [P, ct.c_ulonglong, ct.POINTER(qp_result), P, P, P, P]
    lib.qp_server_poll.restype = I
    lib.qp_server_drain.argtypes = [P, D]
    lib.qp_server_drain.restype = I
    lib.qp_server_get_stats.argtypes = [P, ct.POINTER(qp_server_stats)]
    lib.qp_server_get_stats.restype = I
    lib.qp_server_destroy.argtypes = [P]
    lib.qp_server_destroy.restype = None
    lib.qp_factor_K0.argtypes = [P]
    lib.qp_kf_apply.argtypes = [P, P, P, P, I]
    lib.qp_k0_solve.argtypes = [P, P, P, P, P, I]
    lib.qp_pcg_reduced_solve.argtypes = [P, P, P, P, I, D, I, ct.POINTER(I), ct.POINTER(D), I]
    lib.qp_ipm_solve.argtypes = [P, P, P, P, P, ct.POINTER(D), ct.POINTER(I), ct.POINTER(ct.c_longlong), I]
    lib.qp_get_stats.argtypes = [P, ct.POINTER(qp_stats)]
    lib.qp_device_bytes.argtypes = [P]
    lib.qp_device_bytes.restype = ct.c_size_t
    lib.qp_pcg_bytes_per_iter.argtypes = [P, I]
    lib.qp_pcg_bytes_per_iter.restype = D
    lib.qp_time_pcg_iteration.argtypes = [P, P, I, I, I, ct.POINTER(D), I]
    lib.qp_batch_solve.argtypes = [ct.POINTER(P), I, I, ct.POINTER(qp_result)]
    lib.qp_batch_solve.restype = I
    lib.qp_get_solution.argtypes = [P, P, P, P, P, I]
    lib.qp_get_solution.restype = I
    lib.qp_kf_apply_static.argtypes = [I, I, I, P, P, P, P, P, P, P]
    lib.qp_kf_apply_static.restype = I
    lib.qp_kernel_launches.argtypes = []
    lib.qp_kernel_launches.restype = ct.c_ulonglong
    lib.qp_destroy.argtypes = [P]
    lib.qp_destroy.restype = None
    lib.qp_strerror.argtypes = [I]
    lib.qp_strerror.restype = ct.c_char_p
    for name in ("qp_create", "qp_factor_K0", "qp_kf_apply", "qp_k0_solve", "qp_pcg_reduced_solve",
                 "qp_ipm_solve", "qp_get_stats", "qp_time_pcg_iteration"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


class QPError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {qp_strerror(status)} ({status})")


def _check(st, where, ok=(QP_OK,)):
    if st not in ok:
        raise QPError(st, where)
    return st


def _ptr(a, kind_holder):
    """Raw pointer of a float64 array (numpy host or torch CUDA), recording its kind."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        kind = QP_PTR_HOST
        p = a.ctypes.data
    else:  # torch tensor
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("device tensors must be contiguous float64")
        kind = QP_PTR_DEVICE if a.is_cuda else QP_PTR_HOST
        p = a.data_ptr()
    if kind_holder and kind_holder[0] is not None and kind_holder[0] != kind:
        raise TypeError("mixing host and device arrays in one call")
    if kind_holder is not None:
        kind_holder[0] = kind
    return p


def qp_opts_default() -> qp_opts:
    o = qp_opts()
    load().qp_opts_default(ct.byref(o))
    return o


def qp_strerror(status: int) -> str:
    return load().qp_strerror(int(status)).decode()


def qp_create(H, c, A, b, C, d, opts: qp_opts | None = None):
    """Create a handle (returns an opaque c_void_p).  A/b may be None (m1 = 0)."""
    kh = [None]
    n = int(H.shape[0])
    m1 = 0 if A is None else int(A.shape[0])
    m2 = int(d.shape[0])
    h = ct.c_void_p()
    st = load().qp_create(ct.byref(h), n, m1, m2, _ptr(H, kh), _ptr(c, kh), _ptr(A, kh), _ptr(b, kh),
                          _ptr(C, kh), _ptr(d, kh), ct.byref(opts) if opts is not None else None, kh[0])
    _check(st, "qp_create")
    return h


def qp_create_csr(H, c, A, b, rowptr, colidx, val, d, opts: qp_opts | None = None):
    """qp_create with C in CSR form (host int32 rowptr / colidx, float64 val)."""
    kh = [None]
    n = int(H.shape[0])
    m1 = 0 if A is None else int(A.shape[0])
    m2 = int(d.shape[0])
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    h = ct.c_void_p()
    st = load().qp_create_csr(ct.byref(h), n, m1, m2, _ptr(H, kh), _ptr(c, kh), _ptr(A, kh), _ptr(b, kh),
                              rp.ctypes.data, ci.ctypes.data, _ptr(np.ascontiguousarray(val, dtype=np.float64), kh),
                              _ptr(d, kh), ct.byref(opts) if opts is not None else None, kh[0])
    _check(st, "qp_create_csr")
    return h


def qp_device_bytes_bound(n, m1, m2, opts: qp_opts | None = None) -> int:
    return int(load().qp_device_bytes_bound(int(n), int(m1), int(m2), ct.byref(opts) if opts is not None else None))


def qp_factor_K0(h):
    return _check(load().qp_factor_K0(h), "qp_factor_K0")


def qp_kf_apply(h, D, p, q):
    kh = [None]
    args = (_ptr(D, kh), _ptr(p, kh), _ptr(q, kh))
    return _check(load().qp_kf_apply(h, *args, kh[0]), "qp_kf_apply")


def qp_k0_solve(h, u, w, a, b=None):
    kh = [None]
    args = (_ptr(u, kh), _ptr(w, kh), _ptr(a, kh), _ptr(b, kh))
    return _check(load().qp_k0_solve(h, *args, kh[0]), "qp_k0_solve")


def qp_pcg_reduced_solve(h, D, rhs, dnu, precond=QP_PC_AUTO, tol=1e-8, maxit=1000, allow_maxit=False):
    """Returns (status, iterations, relative residual)."""
    kh = [None]
    args = (_ptr(D, kh), _ptr(rhs, kh), _ptr(dnu, kh))
    it = ct.c_int(0)
    rel = ct.c_double(0)
    st = load().qp_pcg_reduced_solve(h, *args, int(precond), float(tol), int(maxit), ct.byref(it),
                                     ct.byref(rel), kh[0])
    _check(st, "qp_pcg_reduced_solve", ok=(QP_OK, QP_EMAXIT) if allow_maxit else (QP_OK,))
    return st, it.value, rel.value


def qp_ipm_solve(h, x=None, lam=None, nu=None, s=None, allow=(QP_OK,)):
    """Returns (status, objective, ipm_iters, pcg_iters_total)."""
    kh = [None]
    args = (_ptr(x, kh), _ptr(lam, kh), _ptr(nu, kh), _ptr(s, kh))
    kind = kh[0] if kh[0] is not None else QP_PTR_HOST
    obj = ct.c_double(0)
    it = ct.c_int(0)
    pit = ct.c_longlong(0)
    st = load().qp_ipm_solve(h, *args, ct.byref(obj), ct.byref(it), ct.byref(pit), kind)
    _check(st, "qp_ipm_solve", ok=allow)
    return st, obj.value, it.value, pit.value


def qp_get_stats(h) -> dict:
    s = qp_stats()
    _check(load().qp_get_stats(h, ct.byref(s)), "qp_get_stats")
    return s.as_dict()


def qp_device_bytes(h) -> int:
    return int(load().qp_device_bytes(h))


def qp_pcg_bytes_per_iter(h, precond=QP_PC_AUTO) -> float:
    return float(load().qp_pcg_bytes_per_iter(h, int(precond)))


def qp_time_pcg_iteration(h, D, precond=QP_PC_AUTO, warmup=8, iters=64) -> float:
    kh = [None]
    pD = _ptr(D, kh)
    ms = ct.c_double(0)
    _check(load().qp_time_pcg_iteration(h, pD, int(precond), int(warmup), int(iters), ct.byref(ms), kh[0]),
           "qp_time_pcg_iteration")
    return ms.value


def qp_kf_apply_static(C, WH, Gt, D, p, q, stream=None):
    """q = K_F p through the no-allocation entry point (all torch CUDA float64
    tensors; Gt may be None when m1 = 0).  Enqueued on `stream` (a torch stream
    or None for the default stream); returns the status.

    The C side receives raw pointers and cannot check sizes, so every shape and
    device is checked here before the call: C (m2, n), WH (n, n), Gt (m1, n),
    D, p, q (m2,), all on one CUDA device that is the current device and the
    stream's device."""
    if C.dim() != 2:
        raise ValueError("C must be a matrix (m2, n)")
    m2, n = int(C.shape[0]), int(C.shape[1])
    m1 = 0 if Gt is None else int(Gt.shape[0])
    if tuple(WH.shape) != (n, n):
        raise ValueError(f"WH must be ({n}, {n}), got {tuple(WH.shape)}")
    if Gt is not None and (Gt.dim() != 2 or int(Gt.shape[1]) != n):
        raise ValueError(f"Gt must be (m1, {n}), got {tuple(Gt.shape)}")
    for name, v in (("D", D), ("p", p), ("q", q)):
        if v.dim() != 1 or int(v.shape[0]) != m2:
            raise ValueError(f"{name} must be ({m2},), got {tuple(v.shape)}")
    tensors = [a for a in (C, WH, Gt, D, p, q) if a is not None]
    if not all(a.is_cuda for a in tensors):
        raise TypeError("qp_kf_apply_static takes CUDA tensors")
    import torch
    devs = {a.device.index for a in tensors}
    cur = torch.cuda.current_device()
    if devs != {cur}:
        raise ValueError(f"all tensors must be on the current device cuda:{cur}, got {sorted(devs)}")
    if stream is not None and stream.device.index != cur:
        raise ValueError(f"stream is on cuda:{stream.device.index}, the tensors on cuda:{cur}")
    kh = [None]
    args = [_ptr(C, kh), _ptr(WH, kh), _ptr(Gt, kh), _ptr(D, kh), _ptr(p, kh), _ptr(q, kh)]
    sp = None if stream is None else stream.cuda_stream
    return _check(load().qp_kf_apply_static(n, m1, m2, *args, sp), "qp_kf_apply_static")


def qp_batch_solve(handles, max_concurrent=0):
    """Solve many handles concurrently; returns (status, [result dicts])."""
    n = len(handles)
    arr = (ct.c_void_p * n)(*[h.value if isinstance(h, ct.c_void_p) else h for h in handles])
    res = (qp_result * n)()
    st = load().qp_batch_solve(arr, n, int(max_concurrent), res)
    return st, [r.as_dict() for r in res]


def qp_get_solution(h, x=None, lam=None, nu=None, s=None):
    kh = [None]
    args = (_ptr(x, kh), _ptr(lam, kh), _ptr(nu, kh), _ptr(s, kh))
    return _check(load().qp_get_solution(h, *args, kh[0] if kh[0] is not None else QP_PTR_HOST),
                  "qp_get_solution")


def qp_kernel_launches() -> int:
    return int(load().qp_kernel_launches())


def qp_destroy(h):
    if h:
        load().qp_destroy(h)


class QP:
    """Owning wrapper of a handle: QP(qpgen.QP or arrays, opts)."""

    def __init__(self, H, c, A, b, C, d, opts: qp_opts | None = None):
        self.h = qp_create(H, c, A, b, C, d, opts)
        self.n, self.m1, self.m2 = int(H.shape[0]), (0 if A is None else int(A.shape[0])), int(d.shape[0])

    @classmethod
    def from_qpgen(cls, q, opts=None):
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        A = c(q.A) if q.m1 else None
        b = c(q.b) if q.m1 else None
        return cls(c(q.H), c(q.c), A, b, c(q.C_dense()), c(q.d), opts)

    def factor(self):
        qp_factor_K0(self.h)
        return self

    def close(self):
        if self.h:
            qp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving layer: submit QPs (qpgen.QP), poll or drain their results.

    Server(budget_bytes, max_slots, opts); submit(q) -> ticket;
    poll(ticket) -> None while pending, else (result dict, x); drain(timeout_ms);
    stats() -> dict; close()."""

    def __init__(self, budget_bytes=0, max_slots=0, opts: qp_opts | None = None):
        self.h = ct.c_void_p()
        _check(load().qp_server_create(ct.byref(self.h), int(budget_bytes), int(max_slots),
                                       ct.byref(opts) if opts is not None else None), "qp_server_create")
        self._dims = {}

    def submit(self, q) -> int:
        keep = []

        def p(a, dtype=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dtype)
            keep.append(a)
            return a.ctypes.data

        pr = qp_problem()
        pr.n, pr.m1, pr.m2 = q.n, q.m1, q.m2
        pr.H, pr.c, pr.d = p(q.H), p(q.c), p(q.d)
        pr.A = p(q.A) if q.m1 else None
        pr.b = p(q.b) if q.m1 else None
        if q.C_csr is not None:
            rp, ci, val = q.C_csr
            pr.C_rowptr, pr.C_colidx, pr.C_val = p(rp, np.int32), p(ci, np.int32), p(val)
            pr.C = None
        else:
            pr.C = p(q.C)
        t = ct.c_ulonglong(0)
        _check(load().qp_server_submit(self.h, ct.byref(pr), ct.byref(t)), "qp_server_submit")
        self._dims[t.value] = (q.n, q.m1, q.m2)
        return t.value

    def poll(self, ticket, want_x=True):
        n = self._dims.get(ticket, (0, 0, 0))[0]
        want_x = want_x and n > 0
        r = qp_result()
        x = np.zeros(n) if want_x else None
        st = load().qp_server_poll(self.h, ct.c_ulonglong(ticket), ct.byref(r),
                                   x.ctypes.data if want_x else None, None, None, None)
        if st == QP_EAGAIN:
            return None
        _check(st, "qp_server_poll")
        self._dims.pop(ticket, None)
        return r.as_dict(), x

    def drain(self, timeout_ms=-1.0):
        return _check(load().qp_server_drain(self.h, float(timeout_ms)), "qp_server_drain")

    def stats(self) -> dict:
        s = qp_server_stats()
        _check(load().qp_server_get_stats(self.h, ct.byref(s)), "qp_server_get_stats")
        return s.as_dict()

    def close(self):
        if self.h:
            load().qp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
