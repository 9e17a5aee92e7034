"""Python binding of the FRKC2 C ABI (``include/frkc2.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of
the method: plans are built by the library's host code and every stage runs in the CUDA
kernels of ``libfrkc2.so``.  Device buffers are torch CUDA tensors (the library reads and
writes their memory in place); streams are torch streams.  There is no CPU fallback: if
the library has not been built, importing this module raises ``ImportError``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# FRKC2_DEBUG_BOUNDS=1 loads the bounds-checking build (every kernel index checked against
# its array, a violation latched as EBOUNDS and the access skipped)
_DEBUG = os.environ.get("FRKC2_DEBUG_BOUNDS", "0") not in ("", "0")
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                         "libfrkc2_debug.so" if _DEBUG else "libfrkc2.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"FRKC2 CUDA library not built ({_LIB_PATH}); run paper_1702_03818_gb300.build"
                      + (" with debug=True" if _DEBUG else ""))
_lib = C.CDLL(_LIB_PATH)

OK, EINVAL, EUNSTABLE, EPLAN, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED, EBOUNDS = range(10)
BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
KAPPA_CONST, KAPPA_FIELD, KAPPA_POWER = 0, 1, 2
FP64, FP32, MIXED, DFLOAT = 0, 1, 2, 3
PLAN_STRICT, PLAN_GREEDY, PLAN_LEBEDEV, PLAN_PAIRED, PLAN_ORDER4 = 1, 2, 4, 8, 16
PRECISION = {"fp64": FP64, "fp32": FP32, "mixed": MIXED, "dfloat": DFLOAT}
PROBE_PACKED = 16  # frkc2_fma_probe: packed two-lane FP32 FMAs
BC = {"periodic": BC_PERIODIC, "dirichlet": BC_DIRICHLET, "neumann": BC_NEUMANN}
KAPPA = {"const": KAPPA_CONST, "field": KAPPA_FIELD, "power": KAPPA_POWER}


class frkc2_problem(C.Structure):
    _fields_ = [("ndim", C.c_int), ("bc", C.c_int), ("kappa_kind", C.c_int), ("precision", C.c_int),
                ("n", C.c_int64 * 3), ("dx", C.c_double), ("kappa_c", C.c_double),
                ("kappa_p", C.c_double), ("kappa", C.c_void_p)]


class frkc2_bruss_problem(C.Structure):
    _fields_ = [("bc", C.c_int), ("precision", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64),
                ("dx", C.c_double), ("D", C.c_double), ("A", C.c_double), ("B", C.c_double)]


class frkc2_adaptive_stats(C.Structure):
    _fields_ = [("accepted", C.c_int), ("rejected", C.c_int), ("t", C.c_double), ("dt_last", C.c_double),
                ("err_last", C.c_double)]


class frkc2_tuning(C.Structure):
    _fields_ = [("k", C.c_int), ("tile_x", C.c_int), ("tile_y", C.c_int), ("tile_z", C.c_int),
                ("kernel", C.c_int), ("wait_limit", C.c_longlong), ("fault_inject", C.c_int)]


_P = C.c_void_p
_sig = {
    "frkc2_plan": (C.c_int, [C.c_int, C.c_double, C.c_uint, C.POINTER(_P)]),
    "frkc2_plan_from_steps": (C.c_int, [C.c_int, _P, _P, C.POINTER(_P)]),
    "frkc2_plan_info": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "frkc2_plan_destroy": (None, [_P]),
    "frkc2_plan_rounding_gain": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "frkc2_precision_policy": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_int, C.c_double,
                                         C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "frkc2_plan_auto": (C.c_int, [C.c_int, C.POINTER(frkc2_problem), C.c_int, C.c_double, C.POINTER(_P),
                                  C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "frkc2_rho_bound": (C.c_int, [C.POINTER(frkc2_problem), _P, _P, _P]),
    "frkc2_workspace_size": (C.c_int, [C.POINTER(frkc2_problem), C.POINTER(frkc2_tuning), C.POINTER(C.c_size_t)]),
    "frkc2_workspace_reset": (C.c_int, [_P, _P]),
    "frkc2_workspace_status": (C.c_int, [_P, _P]),
    "frkc2_step": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_double, _P, _P,
                             C.c_size_t, C.POINTER(frkc2_tuning), _P]),
    "frkc2_step_noalloc": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_double, _P, _P]),
    "frkc2_stages": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_int, _P, _P, C.c_size_t,
                               _P]),
    "frkc2_adaptive_workspace_size": (C.c_int, [C.POINTER(frkc2_problem), C.POINTER(frkc2_tuning),
                                                C.POINTER(C.c_size_t)]),
    "frkc2_step_adaptive": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_double, C.c_double,
                                      C.c_double, _P, _P, C.c_size_t, C.POINTER(frkc2_tuning),
                                      C.POINTER(frkc2_adaptive_stats), _P]),
    "frkc2_adjoint_workspace_size": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_int, C.c_int,
                                               C.POINTER(C.c_size_t)]),
    "frkc2_adjoint": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_int, _P, _P, _P,
                                _P, _P, C.c_size_t, _P]),
    "frkc2_adjoint_forward": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_int, _P, _P,
                                        _P, C.c_size_t, _P]),
    "frkc2_adjoint_backward": (C.c_int, [_P, C.POINTER(frkc2_problem), C.c_double, C.c_int, C.c_int, _P, _P,
                                         _P, _P, C.c_size_t, _P]),
    "frkc2_batch_workspace_size": (C.c_int, [C.c_int, _P, C.POINTER(frkc2_problem), _P,
                                             C.POINTER(frkc2_tuning), C.POINTER(C.c_size_t)]),
    "frkc2_batch_prepare": (C.c_int, [C.c_int, _P, C.POINTER(frkc2_problem), _P, _P, _P,
                                      C.POINTER(frkc2_tuning), _P, C.c_size_t, _P]),
    "frkc2_batch_launch": (C.c_int, [_P, _P]),
    "frkc2_step_batched": (C.c_int, [C.c_int, _P, C.POINTER(frkc2_problem), _P, _P, _P,
                                     C.POINTER(frkc2_tuning), _P, C.c_size_t, _P]),
    "frkc2_bruss_workspace_size": (C.c_int, [C.POINTER(frkc2_bruss_problem), C.POINTER(C.c_size_t)]),
    "frkc2_bruss_rho_bound": (C.c_int, [C.POINTER(frkc2_bruss_problem), _P, _P, _P, _P, C.c_size_t, _P]),
    "frkc2_bruss_step": (C.c_int, [_P, C.POINTER(frkc2_bruss_problem), C.c_double, C.c_int, C.c_double, _P, _P,
                                   _P, C.c_size_t, C.POINTER(frkc2_tuning), _P]),
    "frkc2_fma_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P]),
    "frkc2_status_string": (C.c_char_p, [C.c_int]),
    "frkc2_launch_count": (C.c_longlong, []),
}
EXPORTED = sorted(_sig)
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name, None)
    if _f is not None:
        _f.restype = _res
        _f.argtypes = _args


class Frkc2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {frkc2_status_string(status)} (status {status})")


def _check(st: int, where: str):
    if st != OK:
        raise Frkc2Error(st, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return _P(t)
    return _P(t.data_ptr())


def frkc2_status_string(status: int) -> str:
    return _lib.frkc2_status_string(int(status)).decode()


def frkc2_launch_count() -> int:
    return int(_lib.frkc2_launch_count())


class Plan:
    """Owns a ``frkc2_plan_t`` handle."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.frkc2_plan_destroy(self._h)
            self._h = None

    def info(self) -> dict:
        return frkc2_plan_info(self)


def frkc2_plan(s: int, nu: float = 0.0, flags: int = 0) -> Plan:
    h = _P()
    _check(_lib.frkc2_plan(int(s), float(nu), int(flags), C.byref(h)), "frkc2_plan")
    return Plan(h)


def frkc2_plan_from_steps(a) -> Plan:
    a = np.asarray(a, dtype=np.complex128)
    re = np.ascontiguousarray(a.real)
    im = np.ascontiguousarray(a.imag)
    h = _P()
    _check(_lib.frkc2_plan_from_steps(len(a), re.ctypes.data, im.ctypes.data, C.byref(h)),
           "frkc2_plan_from_steps")
    return Plan(h)


def frkc2_plan_info(plan: Plan) -> dict:
    s, n_iter = C.c_int(), C.c_int()
    beta, Q = C.c_double(), C.c_double()
    _check(_lib.frkc2_plan_info(plan.handle, C.byref(s), C.byref(beta), C.byref(Q), C.byref(n_iter),
                                None, None, None), "frkc2_plan_info")
    L = s.value
    re = np.zeros(L)
    im = np.zeros(L)
    order = np.zeros(L, dtype=np.int32)
    _check(_lib.frkc2_plan_info(plan.handle, None, None, None, None, re.ctypes.data, im.ctypes.data,
                                order.ctypes.data), "frkc2_plan_info")
    return dict(s=L, beta=beta.value, Q=Q.value, n_iter=n_iter.value, a=re + 1j * im, order=order)


def frkc2_plan_rounding_gain(plan: Plan) -> float:
    g = C.c_double()
    _check(_lib.frkc2_plan_rounding_gain(plan.handle, C.byref(g)), "frkc2_plan_rounding_gain")
    return g.value


PRECISION_NAME = {v: k for k, v in PRECISION.items()}


def frkc2_precision_policy(plan: Plan, prob: frkc2_problem, nsteps: int, tol: float):
    """Returns (precision name, predicted relative error)."""
    pr, e = C.c_int(), C.c_double()
    _check(_lib.frkc2_precision_policy(plan.handle, C.byref(prob), int(nsteps), float(tol), C.byref(pr),
                                       C.byref(e)), "frkc2_precision_policy")
    return PRECISION_NAME[pr.value], e.value


def frkc2_plan_auto(s: int, prob: frkc2_problem, nsteps: int, tol: float):
    """Returns (Plan, precision name, predicted relative error)."""
    h, pr, e = _P(), C.c_int(), C.c_double()
    _check(_lib.frkc2_plan_auto(int(s), C.byref(prob), int(nsteps), float(tol), C.byref(h), C.byref(pr),
                                C.byref(e)), "frkc2_plan_auto")
    return Plan(h), PRECISION_NAME[pr.value], e.value


def make_problem(ndim: int, n, dx: float, bc="periodic", kappa="field", precision="fp64",
                 kappa_c: float = 1.0, kappa_p: float = 2.5, kappa_field=None) -> frkc2_problem:
    """Fill a ``frkc2_problem``; ``n`` = (nx, ny, nz) with x fastest; ``kappa_field`` a CUDA tensor."""
    p = frkc2_problem()
    p.ndim = int(ndim)
    p.bc = BC[bc] if isinstance(bc, str) else int(bc)
    p.kappa_kind = KAPPA[kappa] if isinstance(kappa, str) else int(kappa)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    nn = list(n) + [1] * (3 - len(n))
    for d in range(3):
        p.n[d] = int(nn[d])
    p.dx = float(dx)
    p.kappa_c = float(kappa_c)
    p.kappa_p = float(kappa_p)
    p.kappa = kappa_field.data_ptr() if kappa_field is not None else None
    p._keep = kappa_field  # keep the tensor alive as long as the struct
    return p


def make_tuning(k: int = 0, tile=(0, 0, 0), kernel: int = 0, wait_limit: int = 0,
                fault_inject: int = 0) -> frkc2_tuning:
    t = frkc2_tuning()
    t.k = int(k)
    t.tile_x, t.tile_y, t.tile_z = (int(v) for v in (list(tile) + [0, 0, 0])[:3])
    t.kernel = int(kernel)
    t.wait_limit = int(wait_limit)
    t.fault_inject = int(fault_inject)
    return t


def frkc2_rho_bound(prob: frkc2_problem, u, rho_dev, stream=None):
    _check(_lib.frkc2_rho_bound(C.byref(prob), _ptr(u), _ptr(rho_dev), _stream_ptr(stream)),
           "frkc2_rho_bound")


def frkc2_workspace_size(prob: frkc2_problem, tune: frkc2_tuning | None = None) -> int:
    b = C.c_size_t()
    _check(_lib.frkc2_workspace_size(C.byref(prob), C.byref(tune) if tune is not None else None,
                                     C.byref(b)), "frkc2_workspace_size")
    return b.value


def frkc2_workspace_reset(ws, stream=None):
    _check(_lib.frkc2_workspace_reset(_ptr(ws), _stream_ptr(stream)), "frkc2_workspace_reset")


def frkc2_workspace_status(ws, stream=None) -> int:
    return int(_lib.frkc2_workspace_status(_ptr(ws), _stream_ptr(stream)))


def frkc2_step(plan: Plan, prob: frkc2_problem, dt: float, nsteps: int, rho: float, u, ws,
               tune: frkc2_tuning | None = None, stream=None):
    _check(_lib.frkc2_step(plan.handle, C.byref(prob), float(dt), int(nsteps), float(rho), _ptr(u),
                           _ptr(ws), ws.numel() * ws.element_size(),
                           C.byref(tune) if tune is not None else None, _stream_ptr(stream)),
           "frkc2_step")


def frkc2_stages(plan: Plan, prob: frkc2_problem, dt: float, l0: int, l1: int, w, ws, stream=None):
    """Stages l0 .. l1-1 of one step on the interleaved complex state w (in place)."""
    _check(_lib.frkc2_stages(plan.handle, C.byref(prob), float(dt), int(l0), int(l1), _ptr(w), _ptr(ws),
                             ws.numel() * ws.element_size(), _stream_ptr(stream)), "frkc2_stages")


def frkc2_adaptive_workspace_size(prob: frkc2_problem, tune: frkc2_tuning | None = None) -> int:
    b = C.c_size_t()
    _check(_lib.frkc2_adaptive_workspace_size(C.byref(prob), C.byref(tune) if tune is not None else None,
                                              C.byref(b)), "frkc2_adaptive_workspace_size")
    return b.value


def frkc2_step_adaptive(plan: Plan, prob: frkc2_problem, t_end: float, tol: float, dt0: float, rho: float, u,
                        ws, tune: frkc2_tuning | None = None, stream=None) -> dict:
    st = frkc2_adaptive_stats()
    _check(_lib.frkc2_step_adaptive(plan.handle, C.byref(prob), float(t_end), float(tol), float(dt0), float(rho),
                                    _ptr(u), _ptr(ws), ws.numel() * ws.element_size(),
                                    C.byref(tune) if tune is not None else None, C.byref(st),
                                    _stream_ptr(stream)), "frkc2_step_adaptive")
    return dict(accepted=st.accepted, rejected=st.rejected, t=st.t, dt_last=st.dt_last, err_last=st.err_last)


def frkc2_step_noalloc(plan: Plan, prob: frkc2_problem, dt: float, nsteps: int, rho: float, u, stream=None):
    """frkc2_step with the library's built-in scratch array instead of a caller workspace."""
    _check(_lib.frkc2_step_noalloc(plan.handle, C.byref(prob), float(dt), int(nsteps), float(rho), _ptr(u),
                                   _stream_ptr(stream)), "frkc2_step_noalloc")


NOALLOC_SCRATCH_BYTES = 16 << 20


def frkc2_adjoint_workspace_size(plan: Plan, prob: frkc2_problem, nsteps: int, ckpt_every: int) -> int:
    b = C.c_size_t()
    _check(_lib.frkc2_adjoint_workspace_size(plan.handle, C.byref(prob), int(nsteps), int(ckpt_every),
                                             C.byref(b)), "frkc2_adjoint_workspace_size")
    return b.value


def frkc2_adjoint(plan: Plan, prob: frkc2_problem, dt: float, nsteps: int, ckpt_every: int, u0, g,
                  dJdu0, dJdkappa, ws, stream=None):
    _check(_lib.frkc2_adjoint(plan.handle, C.byref(prob), float(dt), int(nsteps), int(ckpt_every),
                              _ptr(u0), _ptr(g), _ptr(dJdu0), _ptr(dJdkappa), _ptr(ws),
                              ws.numel() * ws.element_size(), _stream_ptr(stream)), "frkc2_adjoint")


def frkc2_adjoint_forward(plan: Plan, prob: frkc2_problem, dt: float, nsteps: int, ckpt_every: int, u0, uT,
                          ws, stream=None):
    _check(_lib.frkc2_adjoint_forward(plan.handle, C.byref(prob), float(dt), int(nsteps), int(ckpt_every),
                                      _ptr(u0), _ptr(uT), _ptr(ws), ws.numel() * ws.element_size(),
                                      _stream_ptr(stream)), "frkc2_adjoint_forward")


def frkc2_adjoint_backward(plan: Plan, prob: frkc2_problem, dt: float, nsteps: int, ckpt_every: int, g,
                           dJdu0, dJdkappa, ws, stream=None):
    _check(_lib.frkc2_adjoint_backward(plan.handle, C.byref(prob), float(dt), int(nsteps), int(ckpt_every),
                                       _ptr(g), _ptr(dJdu0), _ptr(dJdkappa), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream_ptr(stream)),
           "frkc2_adjoint_backward")


def _batch_arrays(plans, probs, dt, nsteps, u):
    n = len(plans)
    ph = (_P * n)(*[p.handle for p in plans])
    pa = (frkc2_problem * n)(*probs)
    da = (C.c_double * n)(*[float(x) for x in dt]) if dt is not None else None
    na = (C.c_int * n)(*[int(x) for x in nsteps])
    ua = (_P * n)(*[t.data_ptr() for t in u]) if u is not None else None
    return n, ph, pa, da, na, ua


def frkc2_batch_workspace_size(plans, probs, nsteps, tune: frkc2_tuning | None = None) -> int:
    n, ph, pa, _, na, _ = _batch_arrays(plans, probs, None, nsteps, None)
    b = C.c_size_t()
    _check(_lib.frkc2_batch_workspace_size(n, ph, pa, na, C.byref(tune) if tune is not None else None,
                                           C.byref(b)), "frkc2_batch_workspace_size")
    return b.value


def frkc2_batch_prepare(plans, probs, dt, nsteps, u, ws, tune: frkc2_tuning | None = None, stream=None):
    n, ph, pa, da, na, ua = _batch_arrays(plans, probs, dt, nsteps, u)
    _check(_lib.frkc2_batch_prepare(n, ph, pa, da, na, ua, C.byref(tune) if tune is not None else None,
                                    _ptr(ws), ws.numel() * ws.element_size(), _stream_ptr(stream)),
           "frkc2_batch_prepare")


def frkc2_batch_launch(ws, stream=None):
    _check(_lib.frkc2_batch_launch(_ptr(ws), _stream_ptr(stream)), "frkc2_batch_launch")


def frkc2_step_batched(plans, probs, dt, nsteps, u, ws, tune: frkc2_tuning | None = None, stream=None):
    n, ph, pa, da, na, ua = _batch_arrays(plans, probs, dt, nsteps, u)
    _check(_lib.frkc2_step_batched(n, ph, pa, da, na, ua, C.byref(tune) if tune is not None else None,
                                   _ptr(ws), ws.numel() * ws.element_size(), _stream_ptr(stream)),
           "frkc2_step_batched")


def make_bruss_problem(n, dx: float | None = None, bc="periodic", precision="fp64", D: float = 0.02,
                       A: float = 1.0, B: float = 3.0) -> frkc2_bruss_problem:
    """Fill a ``frkc2_bruss_problem``; ``n`` = (nx, ny) or one side; dx defaults to 1/nx."""
    nx, ny = (n, n) if isinstance(n, int) else (int(n[0]), int(n[1]))
    p = frkc2_bruss_problem()
    p.bc = BC[bc] if isinstance(bc, str) else int(bc)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.nx, p.ny = int(nx), int(ny)
    p.dx = float(dx) if dx is not None else 1.0 / nx
    p.D, p.A, p.B = float(D), float(A), float(B)
    return p


def frkc2_bruss_workspace_size(prob: frkc2_bruss_problem) -> int:
    b = C.c_size_t()
    _check(_lib.frkc2_bruss_workspace_size(C.byref(prob), C.byref(b)), "frkc2_bruss_workspace_size")
    return b.value


def frkc2_bruss_rho_bound(prob: frkc2_bruss_problem, v, w, rho_dev, ws, stream=None):
    _check(_lib.frkc2_bruss_rho_bound(C.byref(prob), _ptr(v), _ptr(w), _ptr(rho_dev), _ptr(ws),
                                      ws.numel() * ws.element_size(), _stream_ptr(stream)),
           "frkc2_bruss_rho_bound")


def frkc2_bruss_step(plan: Plan, prob: frkc2_bruss_problem, dt: float, nsteps: int, rho: float, v, w, ws,
                     tune: frkc2_tuning | None = None, stream=None):
    _check(_lib.frkc2_bruss_step(plan.handle, C.byref(prob), float(dt), int(nsteps), float(rho), _ptr(v), _ptr(w),
                                 _ptr(ws), ws.numel() * ws.element_size(),
                                 C.byref(tune) if tune is not None else None, _stream_ptr(stream)),
           "frkc2_bruss_step")


def frkc2_fma_probe(precision: str, blocks: int, iters: int, out, stream=None):
    """FMA throughput probe (blocks x 256 threads x iters x 8 FMAs); the caller times it.
    ``precision``: "fp64", "fp32", or "fp32x2" (packed two-lane FP32 FMAs)."""
    code = (PRECISION["fp32"] | PROBE_PACKED) if precision == "fp32x2" else PRECISION[precision]
    _check(_lib.frkc2_fma_probe(code, int(blocks), int(iters), _ptr(out), _stream_ptr(stream)),
           "frkc2_fma_probe")


def library_path() -> str:
    return _LIB_PATH
