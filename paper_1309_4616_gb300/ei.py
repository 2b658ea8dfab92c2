"""Python binding of the C ABI in include/ei.h (ctypes; argument marshalling only).

Every step of the computation runs in libei.so; this module converts torch
tensors to device pointers and status codes to exceptions.  It fails loudly
when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_LIB = None
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libei.so")

OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM, \
    ERR_STATE = range(8)
BC_DIRICHLET0, BC_NEUMANN0 = 0, 1
PREC_F64, PREC_F32 = 0, 1
ARITH_DF, ARITH_NATIVE_F64 = 0, 1
EXP_EULER, EXP_ROSENBROCK = 0, 1
NONLIN_NONE, NONLIN_LOGISTIC, NONLIN_COMBUSTION, NONLIN_COMBUSTION_FAST = 0, 1, 2, 3
STATS_MAX_SUBSTEPS = 64
MLP_INPUTS, MLP_OUTPUTS, MLP_PARAMS, MLP_MAX_Q = 12, 2, 9282, 12

# every symbol include/ei.h declares
EXPORTS = [
    "ei_create", "ei_destroy", "ei_set_stream", "ei_set_operator_stencil",
    "ei_set_operator_csr", "ei_estimate_spectrum", "ei_phi_apply", "ei_step",
    "ei_step_host", "ei_leja_points", "ei_divided_differences", "ei_schedule",
    "ei_status_string", "ei_estimate_spectrum_stencil_noalloc",
    "ei_batch_create", "ei_batch_offsets", "ei_batch_phi1", "ei_batch_destroy",
    "ei_mlp_create", "ei_mlp_destroy", "ei_mlp_set_params", "ei_mlp_get_params",
    "ei_mlp_set_decision", "ei_mlp_get_decision", "ei_mlp_forward", "ei_mlp_loss_grad",
    "ei_mlp_train_step", "ei_set_schedule_model", "ei_batch_set_schedule_model",
    "ei_nonlinearity", "ei_set_dirichlet_values", "ei_phi_apply_imag",
    "ei_divided_differences_imag", "ei_schedule_imag", "ei_batch_set_wait_limit",
]


class Options(C.Structure):
    _fields_ = [("m_max", C.c_int), ("arith", C.c_int), ("fixed_s", C.c_int),
                ("profile", C.c_int), ("single_iter", C.c_int), ("tile_rows", C.c_int),
                ("learned", C.c_int), ("no_restart", C.c_int), ("csr_lanes", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("s", C.c_int),
                ("restarts", C.c_int), ("matvecs", C.c_int), ("degree_sum", C.c_int),
                ("degree_max", C.c_int), ("m_sched", C.c_int),
                ("degrees", C.c_int * STATS_MAX_SUBSTEPS), ("launches", C.c_int),
                ("newton_timed", C.c_int), ("newton_fused", C.c_int),
                ("newton_ms", C.c_double), ("learned", C.c_int), ("learned_s", C.c_int),
                ("learned_m", C.c_int), ("learned_pad", C.c_int),
                ("features", C.c_double * MLP_INPUTS), ("arith_used", C.c_int),
                ("p_rechecks", C.c_int), ("newton_bounded", C.c_int), ("coef_table", C.c_int)]

    def degree_list(self):
        return [int(self.degrees[i]) for i in range(min(self.s, STATS_MAX_SUBSTEPS))]

    def as_dict(self):
        return {"alpha": self.alpha, "beta": self.beta, "s": self.s, "restarts": self.restarts,
                "matvecs": self.matvecs, "degree_sum": self.degree_sum,
                "degree_max": self.degree_max, "m_sched": self.m_sched,
                "degrees": self.degree_list(), "launches": self.launches,
                "newton_timed": self.newton_timed, "newton_fused": self.newton_fused,
                "newton_ms": self.newton_ms, "learned": self.learned,
                "learned_s": self.learned_s, "learned_m": self.learned_m,
                "arith_used": self.arith_used, "p_rechecks": self.p_rechecks,
                "newton_bounded": self.newton_bounded, "coef_table": self.coef_table}

    def feature_list(self):
        return [float(self.features[i]) for i in range(MLP_INPUTS)]


class MlpDecision(C.Structure):
    _fields_ = [("z_min", C.c_double), ("rho_m", C.c_double), ("delta_m", C.c_double),
                ("q_max", C.c_int), ("pad", C.c_int)]


class BatchProblem(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("dx", C.c_double), ("dy", C.c_double),
                ("D", C.c_double), ("bx", C.c_double), ("by", C.c_double), ("c", C.c_double),
                ("bc", C.c_int * 4), ("h", C.c_double)]


class BatchStats(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("s", C.c_int),
                ("degree_sum", C.c_int), ("restarts", C.c_int), ("tile_rows", C.c_int),
                ("learned", C.c_int), ("pad", C.c_int)]


class EIError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        vp, i64p, dp, ip = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.ei_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, vp]
        L.ei_destroy.argtypes = [vp]
        L.ei_destroy.restype = None
        L.ei_set_stream.argtypes = [vp, vp]
        L.ei_set_operator_stencil.argtypes = [vp, C.c_int, i64p, dp, vp, C.c_double,
                                              C.POINTER(C.c_void_p), dp, vp, C.c_double, ip,
                                              C.c_int]
        L.ei_set_operator_csr.argtypes = [vp, C.c_int64, C.c_int64, vp, vp, vp, vp, C.c_int]
        L.ei_estimate_spectrum.argtypes = [vp, dp, dp]
        L.ei_phi_apply.argtypes = [vp, C.c_int, C.c_double, vp, vp, C.c_double,
                                   C.POINTER(Options), C.POINTER(Stats)]
        L.ei_phi_apply_imag.argtypes = L.ei_phi_apply.argtypes
        L.ei_divided_differences_imag.argtypes = [C.c_int, C.c_double, C.c_double,
                                                  C.c_double, C.c_int, dp]
        L.ei_schedule_imag.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_int, ip, ip]
        L.ei_step.argtypes = [vp, C.c_int, C.c_double, vp, C.c_int, C.c_double,
                              C.POINTER(Options), C.POINTER(Stats)]
        L.ei_step_host.argtypes = L.ei_step.argtypes
        L.ei_leja_points.argtypes = [C.c_int, dp]
        L.ei_divided_differences.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                             C.c_int, dp]
        L.ei_schedule.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_int, ip, ip]
        L.ei_estimate_spectrum_stencil_noalloc.argtypes = [
            C.c_int, vp, C.c_int, i64p, dp, vp, C.c_double, C.POINTER(C.c_void_p), dp, vp,
            C.c_double, ip, C.c_int, dp, dp]
        L.ei_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int,
                                      C.POINTER(BatchProblem), C.c_int, C.c_double,
                                      C.POINTER(Options)]
        L.ei_batch_offsets.argtypes = [vp, i64p]
        L.ei_batch_phi1.argtypes = [vp, vp, vp, vp, C.POINTER(BatchStats)]
        L.ei_batch_destroy.argtypes = [vp]
        L.ei_batch_destroy.restype = None
        fp = C.POINTER(C.c_float)
        L.ei_mlp_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, vp]
        L.ei_mlp_destroy.argtypes = [vp]
        L.ei_mlp_destroy.restype = None
        L.ei_mlp_set_params.argtypes = [vp, fp]
        L.ei_mlp_get_params.argtypes = [vp, fp]
        L.ei_mlp_set_decision.argtypes = [vp, C.POINTER(MlpDecision)]
        L.ei_mlp_get_decision.argtypes = [vp, C.POINTER(MlpDecision)]
        L.ei_mlp_forward.argtypes = [vp, vp, C.c_int64, vp]
        L.ei_mlp_loss_grad.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_double, C.c_double, dp,
                                       vp]
        L.ei_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_double, C.c_double,
                                        C.c_double, dp]
        L.ei_set_schedule_model.argtypes = [vp, vp]
        L.ei_batch_set_schedule_model.argtypes = [vp, vp]
        L.ei_batch_set_wait_limit.argtypes = [vp, C.c_int64]
        L.ei_nonlinearity.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, vp, vp, vp, vp]
        L.ei_set_dirichlet_values.argtypes = [vp, C.POINTER(vp)]
        L.ei_status_string.argtypes = [C.c_int]
        L.ei_status_string.restype = C.c_char_p
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("ei_destroy", "ei_status_string", "ei_batch_destroy",
                            "ei_mlp_destroy"):
                f.restype = C.c_int
        _LIB = L
    return _LIB


def status_string(st):
    return lib().ei_status_string(int(st)).decode()


def _check(st, where):
    if st != OK:
        raise EIError(st, where)


# ---- host-side pieces ------------------------------------------------------
def leja_points(m=100):
    import numpy as np
    out = np.zeros(m + 1)
    _check(lib().ei_leja_points(m, out.ctypes.data_as(C.POINTER(C.c_double))), "ei_leja_points")
    return out


def divided_differences(k, tau, c, gamma, m=100):
    import numpy as np
    out = np.zeros(m + 1)
    _check(lib().ei_divided_differences(k, tau, c, gamma, m,
                                        out.ctypes.data_as(C.POINTER(C.c_double))),
           "ei_divided_differences")
    return out


def divided_differences_imag(k, tau, c, gamma, m=100):
    """d_j of f(xi) = phi_k(-i tau (c + gamma xi)), complex (numpy complex128)."""
    import numpy as np
    out = np.zeros(2 * (m + 1))
    _check(lib().ei_divided_differences_imag(k, tau, c, gamma, m,
                                             out.ctypes.data_as(C.POINTER(C.c_double))),
           "ei_divided_differences_imag")
    return out[0::2] + 1j * out[1::2]


def schedule_imag(k, h, c, gamma, tol, m_max=100):
    s, m = C.c_int(0), C.c_int(0)
    _check(lib().ei_schedule_imag(k, h, c, gamma, tol, m_max, C.byref(s), C.byref(m)),
           "ei_schedule_imag")
    return s.value, m.value


def schedule(k, h, c, gamma, tol, m_max=100):
    s, m = C.c_int(0), C.c_int(0)
    _check(lib().ei_schedule(k, h, c, gamma, tol, m_max, C.byref(s), C.byref(m)), "ei_schedule")
    return s.value, m.value


def nonlinearity(kind, u, g, dg=None, arith=ARITH_DF, stream=None):
    """g = g(u) and, if dg is given, dg = g'(u), pointwise on the device
    (ei_nonlinearity); u, g, dg contiguous CUDA float64 or float32 tensors of
    one size.  Queued on `stream` (default: the current stream)."""
    import torch
    dt = u.dtype
    if dt not in (torch.float64, torch.float32):
        raise ValueError("u: float64 or float32 expected")
    prec = PREC_F64 if dt == torch.float64 else PREC_F32
    n = u.numel()
    if stream is None:
        stream = torch.cuda.current_stream(u.device)
    _check(lib().ei_nonlinearity(kind, prec, arith, n, _dev_ptr(u, dt, n, "u"),
                                 _dev_ptr(g, dt, n, "g"), _dev_ptr(dg, dt, n, "dg"),
                                 C.c_void_p(stream.cuda_stream)), "ei_nonlinearity")


# ---- context ---------------------------------------------------------------
def _dev_ptr(t, dtype, n=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name}: expected {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Context:
    """One library context on one device and stream."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        _check(lib().ei_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)), "ei_create")
        self._h = h
        self._keep = []
        self.prec = PREC_F64
        self.n = 0
        self._grid = (0, 0, 0)

    def close(self):
        if getattr(self, "_h", None):
            lib().ei_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dtype(self, prec):
        return self._torch.float64 if prec == PREC_F64 else self._torch.float32

    def set_operator_stencil(self, n, dx, D, b, c=0.0, bc=None, prec=PREC_F64):
        """n = (nx, ny[, nz]); D, each b[e] and c are CUDA tensors (shape [nz,]ny,nx)
        or Python floats (constants)."""
        dim = len(n)
        npts = 1
        for v in n:
            npts *= int(v)
        dt = self._dtype(prec)
        self._grid = tuple(int(v) for v in (list(n) + [1] * (3 - dim)))
        n3 = (C.c_int64 * 3)(*(list(n) + [1] * (3 - dim)))
        dx3 = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - dim)))
        bc = bc if bc is not None else [BC_DIRICHLET0] * (2 * dim)
        bc6 = (C.c_int * 6)(*(list(bc) + [BC_NEUMANN0] * (6 - len(bc))))

        def arr_or_const(x, name):
            if isinstance(x, (int, float)):
                return None, float(x)
            return _dev_ptr(x, dt, npts, name), 0.0

        Dp, Dc = arr_or_const(D, "D")
        bptr = (C.c_void_p * 3)()
        bcst = (C.c_double * 3)()
        for e in range(3):
            if e < dim:
                p_, c_ = arr_or_const(b[e], f"b[{e}]")
                bptr[e] = p_.value if p_ is not None else None
                bcst[e] = c_
        cp, cc = arr_or_const(c, "c")
        self._keep = [D, b, c]
        _check(lib().ei_set_operator_stencil(self._h, dim, n3, dx3, Dp, Dc, bptr, bcst, cp, cc,
                                             bc6, prec), "ei_set_operator_stencil")
        self.prec = prec
        self.n = npts

    def set_operator_csr(self, n, rowptr, col, val, diag=None, prec=PREC_F64):
        torch = self._torch
        dt = self._dtype(prec)
        nnz = int(col.numel())
        self._keep = [rowptr, col, val, diag]
        _check(lib().ei_set_operator_csr(
            self._h, int(n), nnz, _dev_ptr(rowptr, torch.int64, int(n) + 1, "rowptr"),
            _dev_ptr(col, torch.int32, nnz, "col"), _dev_ptr(val, dt, nnz, "val"),
            _dev_ptr(diag, dt, int(n), "diag"), prec), "ei_set_operator_csr")
        self.prec = prec
        self.n = int(n)

    def set_dirichlet_values(self, faces):
        """Inhomogeneous Dirichlet data (ei_set_dirichlet_values): a list of up
        to six device tensors (or None) in the operator's precision, face f of
        the size and index order include/ei.h gives; None clears all."""
        if faces is None:
            _check(lib().ei_set_dirichlet_values(self._h, None), "ei_set_dirichlet_values")
            return
        dt = self._dtype(self.prec)
        nx, ny, nz = self._grid
        size = [ny * nz, ny * nz, nx * nz, nx * nz, nx * ny, nx * ny]
        arr = (C.c_void_p * 6)()
        for f in range(6):
            t = faces[f] if f < len(faces) else None
            arr[f] = _dev_ptr(t, dt, size[f], f"face {f}")
        _check(lib().ei_set_dirichlet_values(self._h, arr), "ei_set_dirichlet_values")

    def estimate_spectrum(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().ei_estimate_spectrum(self._h, C.byref(a), C.byref(b)), "ei_estimate_spectrum")
        return a.value, b.value

    @staticmethod
    def _opts(options):
        if options is None:
            return None
        if isinstance(options, Options):
            return C.byref(options)
        o = Options()
        for k, v in options.items():
            setattr(o, k, v)
        return C.byref(o)

    def _n(self):
        # before set_operator the library itself reports EI_ERR_STATE
        return self.n if self.n > 0 else None

    def phi_apply(self, k, h, v, out, tol, options=None, check=True):
        """Stats of the call; with check=False returns (status, stats) instead
        of raising on an error status."""
        dt = self._dtype(self.prec)
        st = Stats()
        rc = lib().ei_phi_apply(self._h, k, h, _dev_ptr(v, dt, self._n(), "v"),
                                _dev_ptr(out, dt, self._n(), "out"), tol, self._opts(options),
                                C.byref(st))
        if not check:
            return rc, st
        _check(rc, "ei_phi_apply")
        return st

    def phi_apply_imag(self, k, h, v, out, tol, options=None, check=True):
        """out = phi_k(-i h H) v for the context's CSR operator H (real
        symmetric); v, out complex128 (FP64 context) or complex64 (FP32)."""
        dt = self._torch.complex128 if self.prec == PREC_F64 else self._torch.complex64
        st = Stats()
        rc = lib().ei_phi_apply_imag(self._h, k, h, _dev_ptr(v, dt, self._n(), "v"),
                                     _dev_ptr(out, dt, self._n(), "out"), tol,
                                     self._opts(options), C.byref(st))
        if not check:
            return rc, st
        _check(rc, "ei_phi_apply_imag")
        return st

    def step(self, method, h, u, nonlin, tol, options=None, check=True):
        dt = self._dtype(self.prec)
        st = Stats()
        rc = lib().ei_step(self._h, method, h, _dev_ptr(u, dt, self._n(), "u"), nonlin, tol,
                           self._opts(options), C.byref(st))
        if not check:
            return rc, st
        _check(rc, "ei_step")
        return st

    def set_schedule_model(self, model):
        """Use `model` (an Mlp, or None) for calls with options learned = 1."""
        self._model = model
        _check(lib().ei_set_schedule_model(self._h, model._h if model is not None else None),
               "ei_set_schedule_model")

    def step_host(self, method, h, u_host, nonlin, tol, options=None):
        """u_host: a CPU tensor; pinned memory is read and written by the
        kernels directly, other memory is copied."""
        dt = self._dtype(self.prec)
        if u_host.is_cuda or not u_host.is_contiguous() or u_host.dtype != dt or \
                u_host.numel() != self.n:
            raise ValueError("u_host: expected a contiguous CPU tensor of the operator's size")
        st = Stats()
        _check(lib().ei_step_host(self._h, method, h, C.c_void_p(u_host.data_ptr()), nonlin,
                                  tol, self._opts(options), C.byref(st)), "ei_step_host")
        return st


class Batch:
    """Many independent 2D constant-coefficient problems advanced by one
    persistent launch (ei_batch_*).  problems: objects with n=(nx, ny),
    dx=(dx, dy), D, b=(bx, by), bc (4 codes), h, and optionally c."""

    def __init__(self, problems, prec=PREC_F64, tol=1e-10, device=0, options=None):
        import numpy as np
        self.count = len(problems)
        arr = (BatchProblem * self.count)()
        for i, p in enumerate(problems):
            q = arr[i]
            q.nx, q.ny = int(p.n[0]), int(p.n[1])
            q.dx, q.dy = float(p.dx[0]), float(p.dx[1])
            q.D = float(p.D)
            q.bx, q.by = float(p.b[0]), float(p.b[1])
            q.c = float(getattr(p, "c", 0.0))
            for f in range(4):
                q.bc[f] = int(p.bc[f])
            q.h = float(p.h)
        h = C.c_void_p()
        _check(lib().ei_batch_create(C.byref(h), device, self.count, arr, prec, tol,
                                     Context._opts(options)), "ei_batch_create")
        self._h = h
        self.prec = prec
        off = np.zeros(self.count + 1, dtype=np.int64)
        _check(lib().ei_batch_offsets(self._h, off.ctypes.data_as(C.POINTER(C.c_int64))),
               "ei_batch_offsets")
        self.offsets = off

    def set_schedule_model(self, model):
        """Plan later passes with `model` (an Mlp, or None: the a-priori rule)."""
        self._model = model
        _check(lib().ei_batch_set_schedule_model(self._h, model._h if model is not None
                                                 else None), "ei_batch_set_schedule_model")

    def set_wait_limit(self, limit_us):
        """The persistent kernel's no-progress limit in microseconds (<= 0: 5 s)."""
        _check(lib().ei_batch_set_wait_limit(self._h, int(limit_us)), "ei_batch_set_wait_limit")

    def phi1(self, v, out, stream=None):
        import torch
        dt = torch.float64 if self.prec == PREC_F64 else torch.float32
        n = int(self.offsets[-1])
        if stream is None:
            stream = torch.cuda.current_stream()
        st = (BatchStats * self.count)()
        _check(lib().ei_batch_phi1(self._h, C.c_void_p(stream.cuda_stream),
                                   _dev_ptr(v, dt, n, "v"), _dev_ptr(out, dt, n, "out"), st),
               "ei_batch_phi1")
        return st

    def close(self):
        if getattr(self, "_h", None):
            lib().ei_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The schedule network (ei_mlp_*): parameters and Adam state on the device."""

    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        _check(lib().ei_mlp_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)),
               "ei_mlp_create")
        self._h = h

    def set_params(self, theta):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters, got {t.size}")
        _check(lib().ei_mlp_set_params(self._h, t.ctypes.data_as(C.POINTER(C.c_float))),
               "ei_mlp_set_params")

    def get_params(self):
        import numpy as np
        t = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(lib().ei_mlp_get_params(self._h, t.ctypes.data_as(C.POINTER(C.c_float))),
               "ei_mlp_get_params")
        return t

    def set_decision(self, z_min=0.0, rho_m=0.05, delta_m=2.0, q_max=MLP_MAX_Q):
        d = MlpDecision(z_min=z_min, rho_m=rho_m, delta_m=delta_m, q_max=q_max)
        _check(lib().ei_mlp_set_decision(self._h, C.byref(d)), "ei_mlp_set_decision")

    def get_decision(self):
        d = MlpDecision()
        _check(lib().ei_mlp_get_decision(self._h, C.byref(d)), "ei_mlp_get_decision")
        return {"z_min": d.z_min, "rho_m": d.rho_m, "delta_m": d.delta_m, "q_max": d.q_max}

    def forward(self, x, out):
        import torch
        rows = x.shape[0]
        _check(lib().ei_mlp_forward(self._h, _dev_ptr(x, torch.float32, rows * MLP_INPUTS, "x"),
                                    rows, _dev_ptr(out, torch.float32, rows * MLP_OUTPUTS,
                                                   "out")), "ei_mlp_forward")

    def loss_grad(self, x, y, mask, grad, lam=0.1, kappa=4.0):
        import torch
        rows = x.shape[0]
        loss = C.c_double()
        _check(lib().ei_mlp_loss_grad(
            self._h, _dev_ptr(x, torch.float32, rows * MLP_INPUTS, "x"),
            _dev_ptr(y, torch.float32, rows * MLP_OUTPUTS, "y"),
            _dev_ptr(mask, torch.float32, rows, "mask"), rows, lam, kappa, C.byref(loss),
            _dev_ptr(grad, torch.float32, MLP_PARAMS, "grad")), "ei_mlp_loss_grad")
        return loss.value

    def train_step(self, x, y, mask, lr, lam=0.1, kappa=4.0, want_loss=True):
        import torch
        rows = x.shape[0]
        loss = C.c_double()
        _check(lib().ei_mlp_train_step(
            self._h, _dev_ptr(x, torch.float32, rows * MLP_INPUTS, "x"),
            _dev_ptr(y, torch.float32, rows * MLP_OUTPUTS, "y"),
            _dev_ptr(mask, torch.float32, rows, "mask"), rows, lam, kappa, lr,
            C.byref(loss) if want_loss else None), "ei_mlp_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            lib().ei_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
