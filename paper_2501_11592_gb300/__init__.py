"""GB300 (sm_103a) batched OMP / CLOMP -- Python binding of the C ABI.

The binding only marshals arguments: torch tensors provide device memory and
the current CUDA stream; every step of the solve runs in the library's CUDA
kernels (``_lib/libcs_omp.so``, built by ``paper_2501_11592_gb300.build``).
There is no CPU path: if the library is missing, :func:`load` raises.

Function names follow the C ABI in ``include/cs_omp.h``.  Matrices are
column-major: pass ``A`` as an (m, n) tensor whose columns are contiguous
(e.g. ``torch.from_numpy(np.asfortranarray(A))`` or ``At.t()`` for a
contiguous (n, m) tensor ``At``); other layouts are copied into that layout.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

__all__ = [
    "load", "Plan", "omp_solve", "omp_solve_batched", "clomp_solve", "clomp_solve_batched",
    "omp_solve_batched_host", "clomp_solve_batched_host", "clfit_forward", "clfit_adjoint",
    "clfit_adam_step", "CSError", "SIG_REACHED_K", "SIG_REACHED_TOL", "SIG_MAX_ITER",
    "SIG_DEPENDENT", "SIG_NONFINITE", "SIG_UNSUPPORTED", "library_path", "correlate", "PHASES", "omp_solve_varlen",
    "clomp_solve_varlen", "synthesize", "image_quality", "reconstruct_columnwise", "iht_solve_batched",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_lib", "libcs_omp.so")

CS_OK, CS_EINVAL, CS_ENOMEM, CS_ECUDA, CS_ETIMEOUT, CS_ENOTSUP = 0, -1, -2, -3, -4, -5
SIG_REACHED_K, SIG_REACHED_TOL, SIG_MAX_ITER, SIG_DEPENDENT, SIG_NONFINITE, SIG_UNSUPPORTED = 0, 1, 2, 3, 4, 5
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
FORM = {"gather": 0, "gram": 1}
PHASES = ("setup", "correlation", "select", "fit", "residual", "update", "persist")
OPT_GRAPHS, OPT_FUSE_UPDATE, OPT_PERSIST, OPT_STALL_TEST, OPT_FUSED_OMP, OPT_AUTOTUNE, OPT_TC_TILE = 0, 1, 2, 3, 4, 5, 6
_STATUS_NAMES = {CS_EINVAL: "CS_EINVAL", CS_ENOMEM: "CS_ENOMEM", CS_ECUDA: "CS_ECUDA",
                 CS_ETIMEOUT: "CS_ETIMEOUT", CS_ENOTSUP: "CS_ENOTSUP"}


class CSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class OmpParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("topc", ctypes.c_int32)]


class Instance(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("lda", ctypes.c_int32), ("y", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("support", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("n_iter", ctypes.c_void_p),
                ("res_norm", ctypes.c_void_p), ("sig_status", ctypes.c_void_p)]


class IhtParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("step", ctypes.c_float)]


class ClompParams(ctypes.Structure):
    _fields_ = [("base", OmpParams), ("steps", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("reset_adam_each_iter", ctypes.c_int32), ("form", ctypes.c_int32),
                ("select_threshold", ctypes.c_float), ("tv_weight", ctypes.c_float),
                ("tv_D", ctypes.c_void_p), ("tv_N", ctypes.c_int32), ("tv_ldd", ctypes.c_int32),
                ("image_width", ctypes.c_int32), ("lv_weight", ctypes.c_float), ("lv_eps", ctypes.c_float)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load the CUDA library (raises FileNotFoundError if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise FileNotFoundError(
                f"{_LIB_PATH} is missing; build it with `python -m paper_2501_11592_gb300.build`")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float
        solve_args = [vp, vp, i32, i32, i32, vp, i32, i32, vp, vp, vp, vp, vp]
        L.cs_plan_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32]
        L.cs_plan_destroy.argtypes = [vp]
        L.omp_solve_batched.argtypes = solve_args + [ctypes.POINTER(OmpParams), vp]
        L.omp_solve_batched_host.argtypes = solve_args + [ctypes.POINTER(OmpParams), vp]
        L.clomp_solve_batched.argtypes = solve_args + [ctypes.POINTER(ClompParams), vp]
        L.clomp_solve_batched_host.argtypes = solve_args + [ctypes.POINTER(ClompParams), vp]
        single = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, vp]
        L.omp_solve.argtypes = single + [ctypes.POINTER(OmpParams), vp]
        L.clomp_solve.argtypes = single + [ctypes.POINTER(ClompParams), vp]
        L.clfit_forward.argtypes = [vp, i32, i32, i32, vp, vp, i32, i32, vp, i32, i32, vp, i32, vp, vp]
        L.clfit_adjoint.argtypes = [vp, i32, i32, i32, vp, i32, i32, vp, i32, i32, vp, vp]
        L.clfit_adam_step.argtypes = [vp, i32, i32, i32, vp, vp, i32, i32, vp, i32, i32, vp, vp,
                                      i32, f32, f32, f32, f32, vp, vp]
        L.cs_correlate.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, i32, vp, i32, vp]
        L.cs_plan_set_A_generation.argtypes = [vp, ctypes.c_uint64]
        L.cs_synthesize.argtypes = [vp, i32, i32, i32, vp, vp, vp, i32, i32, vp, i32, vp]
        L.cs_image_quality.argtypes = [vp, vp, i32, i32, i32, f32, vp, vp, vp]
        L.cs_plan_counters.argtypes = [vp, vp, i32, vp]
        L.cs_plan_set_profiling.argtypes = [vp, i32]
        L.cs_plan_profile.argtypes = [vp, vp, vp, i32]
        L.cs_plan_set_option.argtypes = [vp, i32, i32]
        L.cs_plan_autotune_report.argtypes = [vp, ctypes.c_char_p, i32]
        L.cs_plan_autotune_report.restype = ctypes.c_int
        L.omp_solve_varlen.argtypes = [vp, ctypes.POINTER(Instance), i32, ctypes.POINTER(OmpParams), vp]
        L.iht_solve_batched.argtypes = solve_args + [ctypes.POINTER(IhtParams), vp]
        L.iht_solve_batched.restype = ctypes.c_int
        L.clomp_solve_varlen.argtypes = [vp, ctypes.POINTER(Instance), i32, ctypes.POINTER(ClompParams), vp]
        for fn in ("omp_solve_varlen", "clomp_solve_varlen", "cs_plan_set_option", "cs_correlate", "cs_plan_counters", "cs_plan_set_profiling", "cs_plan_profile",
                   "cs_plan_create", "cs_plan_destroy", "omp_solve_batched", "omp_solve_batched_host",
                   "clomp_solve_batched", "clomp_solve_batched_host", "omp_solve", "clomp_solve",
                   "clfit_forward", "clfit_adjoint", "clfit_adam_step"):
            getattr(L, fn).restype = ctypes.c_int
        L.cs_last_error.restype = ctypes.c_char_p
        L.cs_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc):
    if rc != CS_OK:
        raise CSError(rc, load().cs_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*xs):
    """Every given tensor is a CUDA tensor and all are on one device: the
    library reads its arguments on the GPU, where a host address faults."""
    dev = None
    for x in xs:
        if x is None:
            continue
        if not getattr(x, "is_cuda", False):
            raise ValueError("expected CUDA tensors (host arrays go through the *_host entry points)")
        if dev is None:
            dev = x.device
        elif x.device != dev:
            raise ValueError(f"tensors on {dev} and {x.device}: every argument must be on one device")
    return dev


def _colmajor(x, dtype):
    """(rows, cols) tensor with contiguous columns (stride (1, ld)), on its device."""
    torch = _torch()
    _require_cuda(x)
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if x.dtype != dtype:
        x = x.to(dtype)
    if x.stride(0) != 1 or (x.shape[1] > 1 and x.stride(1) < x.shape[0]):
        x = x.t().contiguous().t()
    return x


def _ld(x):
    return max(int(x.stride(1)), int(x.shape[0])) if x.shape[1] > 1 else int(x.shape[0])


class Plan:
    """Device workspace for problems up to (m_max, n_max, batch_max, k_max)."""

    def __init__(self, m_max, n_max, batch_max, k_max):
        L = load()
        h = ctypes.c_void_p()
        _check(L.cs_plan_create(ctypes.byref(h), int(m_max), int(n_max), int(batch_max), int(k_max)))
        self.h = h
        self.dims = (int(m_max), int(n_max), int(batch_max), int(k_max))

    def fits(self, m, n, B, k):
        return m <= self.dims[0] and n <= self.dims[1] and B <= self.dims[2] and k <= self.dims[3]

    def counters(self, reset=False, stream=None):
        """(certificate fallbacks, device error flags); synchronises the stream."""
        import numpy as np
        out = np.zeros(4, np.uint32)
        rc = load().cs_plan_counters(self.h, ctypes.c_void_p(out.ctypes.data), int(bool(reset)),
                                     _stream_ptr(stream))
        if rc not in (CS_OK, CS_ETIMEOUT):
            _check(rc)
        return int(out[0]), int(out[1])

    def set_option(self, option, value):
        _check(load().cs_plan_set_option(self.h, int(option), int(value)))

    def set_A_generation(self, generation):
        """Keep A's preparation for later solves with the same A until the
        generation changes (0: prepare A in every solve).  Change the
        generation whenever A's contents change: a row-major A is copied to a
        temporary column-major buffer whose address can repeat."""
        _check(load().cs_plan_set_A_generation(self.h, int(generation)))

    def autotune_report(self):
        """{size class: chosen configuration index} of the autotuner."""
        buf = ctypes.create_string_buffer(1 << 16)
        _check(load().cs_plan_autotune_report(self.h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            k, _, v = line.rpartition(" -> ")
            out[k] = int(v)
        return out

    def set_profiling(self, enable=True):
        _check(load().cs_plan_set_profiling(self.h, int(bool(enable))))

    def profile(self, reset=True):
        """{phase: (launches, milliseconds)} since the last reset."""
        import numpy as np
        ms = np.zeros(len(PHASES), np.float64)
        n = np.zeros(len(PHASES), np.int64)
        _check(load().cs_plan_profile(self.h, ctypes.c_void_p(ms.ctypes.data),
                                      ctypes.c_void_p(n.ctypes.data), int(bool(reset))))
        return {ph: (int(n[i]), float(ms[i])) for i, ph in enumerate(PHASES)}

    def close(self):
        if self.h is not None and self.h.value:
            load().cs_plan_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plans: dict = {}


def _plan_for(m, n, B, k, plan):
    if plan is not None:
        return plan
    torch = _torch()
    dev = torch.cuda.current_device()
    p = _plans.get(dev)
    if p is None or not p.fits(m, n, B, k):
        if p is not None:
            m, n, B, k = max(m, p.dims[0]), max(n, p.dims[1]), max(B, p.dims[2]), max(k, p.dims[3])
            p.close()
        p = Plan(m, n, B, k)
        _plans[dev] = p
    return p


@dataclass
class Result:
    support: "object"    # (B, k) int32, selection order, -1 = unused
    coef: "object"       # (B, k) float32
    n_iter: "object"     # (B,) int32
    res_norm: "object"   # (B,) float32
    status: "object"     # (B,) int32 (SIG_*)


def _outputs(B, k, device):
    torch = _torch()
    return Result(torch.empty((B, k), dtype=torch.int32, device=device),
                  torch.empty((B, k), dtype=torch.float32, device=device),
                  torch.empty(B, dtype=torch.int32, device=device),
                  torch.empty(B, dtype=torch.float32, device=device),
                  torch.empty(B, dtype=torch.int32, device=device))


def _omp_params(k, tol, max_iter, prec, topc):
    return OmpParams(int(k), float(tol), int(max_iter or 0), PREC[prec], int(topc))


def _clomp_params(k, tol, max_iter, prec, topc, steps, lr, beta1, beta2, eps, reset_adam, form, th=0.0,
                  tv_weight=0.0, D=None, image_width=0, lv_weight=0.0, lv_eps=1e-4):
    Dp, N, ldd = None, 0, 0
    if D is not None:
        N, ldd = int(D.shape[0]), _ld(D)
        Dp = ctypes.c_void_p(D.data_ptr())
    return ClompParams(_omp_params(k, tol, max_iter, prec, topc), int(steps), float(lr), float(beta1),
                       float(beta2), float(eps), int(bool(reset_adam)), FORM[form], float(th),
                       float(tv_weight), Dp, N, ldd, int(image_width), float(lv_weight), float(lv_eps))


def _batched(fn, A, Y, k, params, plan, stream, out):
    torch = _torch()
    A = _colmajor(A, torch.float32)
    Y = _colmajor(Y, torch.float32)
    m, n = A.shape
    B = Y.shape[1]
    if Y.shape[0] != m:
        raise ValueError(f"Y has {Y.shape[0]} rows, A has {m}")
    p = _plan_for(m, n, B, k, plan)
    o = out if out is not None else _outputs(B, k, A.device)
    _require_cuda(A, Y, o.support, o.coef, o.n_iter, o.res_norm, o.status)
    _check(fn(p.h, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), ctypes.c_void_p(Y.data_ptr()), m if B <= 1 else _ld(Y),
              B, ctypes.c_void_p(o.support.data_ptr()), ctypes.c_void_p(o.coef.data_ptr()),
              ctypes.c_void_p(o.n_iter.data_ptr()), ctypes.c_void_p(o.res_norm.data_ptr()),
              ctypes.c_void_p(o.status.data_ptr()), ctypes.byref(params), _stream_ptr(stream)))
    return o


def omp_solve_batched(A, Y, k, tol=0.0, max_iter=None, prec="fp32", topc=8, plan=None,
                      stream=None, out=None) -> Result:
    """Batched plain OMP on the current stream (see include/cs_omp.h)."""
    return _batched(load().omp_solve_batched, A, Y, k, _omp_params(k, tol, max_iter, prec, topc),
                    plan, stream, out)


def clomp_solve_batched(A, Y, k, tol=0.0, max_iter=None, prec="fp32", topc=8, steps=50, lr=1e-2,
                        beta1=0.9, beta2=0.999, eps=1e-8, reset_adam=False, form="gram",
                        plan=None, stream=None, out=None, th=0.0, tv_weight=0.0, D=None,
                        image_width=0, lv_weight=0.0, lv_eps=1e-4) -> Result:
    """Batched CLOMP (structure 1, Adam) on the current stream; th: the
    selection threshold Th (0: one atom per iteration); tv_weight, D: the
    total-variation prior of Eq. 5 on x = D s (D None: x = s); image_width W >= 2:
    the batch is images of W consecutive columns and the prior is that of an
    image (Eq. 6; D with orthonormal columns or None); lv_weight: the local
    variation of Eq. 7 over those images (any D), each window's deviation
    smoothed as sqrt(var + lv_eps^2)."""
    Dt = None if D is None else _colmajor(D, _torch().float32)
    _require_cuda(A, Y, Dt)
    return _batched(load().clomp_solve_batched, A, Y, k,
                    _clomp_params(k, tol, max_iter, prec, topc, steps, lr, beta1, beta2, eps,
                                  reset_adam, form, th, tv_weight, Dt, image_width, lv_weight, lv_eps), plan,
                    stream, out)


def iht_solve_batched(A, Y, k, step, tol=0.0, max_iter=200, plan=None, stream=None, out=None) -> Result:
    """Batched IHT, s <- H_k(s + step A^T r) for max_iter iterations (float32
    correlation); support lists the kept atoms in ascending index order."""
    return _batched(load().iht_solve_batched, A, Y, k, IhtParams(int(k), float(tol), int(max_iter), float(step)),
                    plan, stream, out)


def omp_solve(A, y, k, **kw) -> Result:
    return omp_solve_batched(A, y.reshape(-1, 1), k, **kw)


def clomp_solve(A, y, k, **kw) -> Result:
    return clomp_solve_batched(A, y.reshape(-1, 1), k, **kw)


def _host_batched(fn, A, Y, k, params, plan, stream, out=None):
    """A, Y: float32 numpy arrays in Fortran order (pinned or pageable)."""
    import numpy as np
    A = np.asfortranarray(A, dtype=np.float32)
    Y = np.asfortranarray(Y.reshape(Y.shape[0], -1), dtype=np.float32)
    m, n = A.shape
    B = Y.shape[1]
    p = _plan_for(m, n, B, k, plan)
    if out is None:
        out = dict(support=np.empty((B, k), np.int32), coef=np.empty((B, k), np.float32),
                   n_iter=np.empty(B, np.int32), res_norm=np.empty(B, np.float32),
                   status=np.empty(B, np.int32))
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(fn(p.h, ptr(A), m, n, m, ptr(Y), m, B, ptr(out["support"]), ptr(out["coef"]),
              ptr(out["n_iter"]), ptr(out["res_norm"]), ptr(out["status"]), ctypes.byref(params),
              _stream_ptr(stream)))
    return out


def omp_solve_batched_host(A, Y, k, tol=0.0, max_iter=None, prec="fp32", topc=8, plan=None,
                           stream=None, out=None):
    return _host_batched(load().omp_solve_batched_host, A, Y, k,
                         _omp_params(k, tol, max_iter, prec, topc), plan, stream, out)


def clomp_solve_batched_host(A, Y, k, tol=0.0, max_iter=None, prec="fp32", topc=8, steps=50,
                             lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, reset_adam=False,
                             form="gram", plan=None, stream=None, out=None, th=0.0):
    return _host_batched(load().clomp_solve_batched_host, A, Y, k,
                         _clomp_params(k, tol, max_iter, prec, topc, steps, lr, beta1, beta2, eps,
                                       reset_adam, form, th), plan, stream, out)


def _varlen(fn, instances, params, plan, stream):
    """instances: list of (A (m, n) column-major tensor, y (m,) tensor, k).
    Returns a list of Result (one signal each)."""
    torch = _torch()
    for A, y, _ in instances:
        _require_cuda(A, y)
    if plan is None:
        # instances beyond the kernels' limits are refused per instance
        # (SIG_UNSUPPORTED), so the default plan stops at those limits
        m_max = min(32768, max(int(A.shape[0]) for A, _, _ in instances))
        n_max = max(int(A.shape[1]) for A, _, _ in instances)
        k_max = min(4096, max(int(k) for _, _, k in instances))
        plan = _plan_for(m_max, n_max, 1024, k_max, None)
    keep, outs = [], []
    arr = (Instance * len(instances))()
    for i, (A, y, k) in enumerate(instances):
        A = _colmajor(A, torch.float32)
        y = y.to(torch.float32).contiguous()
        o = _outputs(1, int(k), A.device)
        keep += [A, y]
        outs.append(o)
        arr[i] = Instance(A.data_ptr(), A.shape[0], A.shape[1], _ld(A), y.data_ptr(), int(k),
                          o.support.data_ptr(), o.coef.data_ptr(), o.n_iter.data_ptr(),
                          o.res_norm.data_ptr(), o.status.data_ptr())
    _check(fn(plan.h, arr, len(instances), ctypes.byref(params), _stream_ptr(stream)))
    return outs


def omp_solve_varlen(instances, tol=0.0, max_iter=None, prec="fp32", plan=None, stream=None):
    """Uneven batch of (A, y, k) instances, plain OMP."""
    return _varlen(load().omp_solve_varlen, instances, _omp_params(1, tol, max_iter, prec, 0), plan, stream)


def clomp_solve_varlen(instances, tol=0.0, max_iter=None, prec="fp32", steps=50, lr=1e-2, beta1=0.9,
                       beta2=0.999, eps=1e-8, reset_adam=False, form="gram", plan=None, stream=None):
    """Uneven batch of (A, y, k) instances, CLOMP."""
    return _varlen(load().clomp_solve_varlen, instances,
                   _clomp_params(1, tol, max_iter, prec, 0, steps, lr, beta1, beta2, eps, reset_adam, form),
                   plan, stream)


def correlate(A, R, prec="fp32", plan=None, stream=None):
    """C = A^T R (n x B, column-major) -- the residual-injection layer alone."""
    torch = _torch()
    A = _colmajor(A, torch.float32)
    R = _colmajor(R, torch.float32)
    _require_cuda(A, R)
    m, n = A.shape
    B = R.shape[1]
    p = _plan_for(m, n, B, 1, plan)
    C = torch.empty((B, n), dtype=torch.float32, device=A.device).t()
    _check(load().cs_correlate(p.h, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), ctypes.c_void_p(R.data_ptr()),
                               m if B <= 1 else _ld(R), B, PREC[prec], ctypes.c_void_p(C.data_ptr()), n,
                               _stream_ptr(stream)))
    return C


def synthesize(D, support, coef, n_iter, stream=None, n=None):
    """X[:, b] = D[:, support[b, :n_iter[b]]] @ coef[b, :n_iter[b]]: the
    signals (image columns) from a solve's sparse codes.  D: (N, n);
    support, coef: (B, k); n_iter: (B,).  D None: the dense codes themselves
    (X is n x B; give n).  Returns X (N, B), column-major."""
    torch = _torch()
    if D is None:
        if n is None:
            raise ValueError("synthesize without a basis needs n")
        N = int(n)
        Dp, ldd = None, N
        dev = support.device
    else:
        D = _colmajor(D, torch.float32)
        N, n = D.shape
        Dp, ldd = ctypes.c_void_p(D.data_ptr()), _ld(D)
        dev = D.device
    _require_cuda(D, support, coef, n_iter)
    support = support.to(torch.int32).contiguous()
    coef = coef.to(torch.float32).contiguous()
    n_iter = n_iter.to(torch.int32).contiguous()
    B, k = support.shape
    X = torch.empty((B, N), dtype=torch.float32, device=dev).t()
    _check(load().cs_synthesize(Dp, N, int(n), ldd, ctypes.c_void_p(support.data_ptr()),
                                ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(n_iter.data_ptr()), k, B,
                                ctypes.c_void_p(X.data_ptr()), N, _stream_ptr(stream)))
    return X


def image_quality(X, Xref, W, peak=0.0, stream=None):
    """Per-image PSNR and SSIM of the consecutive H x W images held as the
    columns of X (H rows, count * W columns) against Xref (same layout).
    peak <= 0: each reference's max - min.  Returns (psnr, ssim) tensors."""
    torch = _torch()
    X = _colmajor(X, torch.float32)
    R = _colmajor(Xref, torch.float32)
    _require_cuda(X, R)
    H = X.shape[0]
    if X.shape != R.shape or X.shape[1] % W:
        raise ValueError(f"X {tuple(X.shape)} and Xref {tuple(R.shape)} must match and hold whole H x {W} images")
    if (X.shape[1] > 1 and X.stride(1) != H) or (R.shape[1] > 1 and R.stride(1) != H):
        X = X.t().contiguous().t()
        R = R.t().contiguous().t()
    count = X.shape[1] // W
    psnr = torch.empty(count, dtype=torch.float32, device=X.device)
    ssim = torch.empty(count, dtype=torch.float32, device=X.device)
    _check(load().cs_image_quality(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(R.data_ptr()), H, W, count,
                                   float(peak), ctypes.c_void_p(psnr.data_ptr()), ctypes.c_void_p(ssim.data_ptr()),
                                   _stream_ptr(stream)))
    return psnr, ssim


def reconstruct_columnwise(A, D, Y, k, W, ref=None, algo="clomp", prec="bf16", peak=0.0, plan=None,
                           stream=None, image_prior=False, **kw):
    """Column-wise 2D reconstruction (Eq. 3 applied to the columns of
    images): solve every measured column y = A s with A = M D, synthesise the
    image columns x = D s, and, given the reference images, their PSNR and
    SSIM.  Y: (m, count * W); tv_weight > 0 (CLOMP) adds the total-variation
    prior of Eq. 5 on each column x = D s, or with image_prior=True that of
    the whole image (Eq. 6); lv_weight > 0 adds the local variation of Eq. 7
    over each image.  Returns dict(X, result, psnr, ssim)."""
    fn = clomp_solve_batched if algo == "clomp" else omp_solve_batched
    if algo == "clomp" and (kw.get("tv_weight", 0.0) > 0.0 or kw.get("lv_weight", 0.0) > 0.0):
        kw.setdefault("D", D)       # the priors act on the image columns x = D s
        if image_prior or kw.get("lv_weight", 0.0) > 0.0:
            kw.setdefault("image_width", W)
    res = fn(A, Y, k, prec=prec, plan=plan, stream=stream, **kw)
    X = synthesize(D, res.support, res.coef, res.n_iter, stream=stream)
    out = dict(X=X, result=res, psnr=None, ssim=None)
    if ref is not None:
        out["psnr"], out["ssim"] = image_quality(X, ref, W, peak=peak, stream=stream)
    return out


def clfit_forward(A, S, Sv, Y, stream=None):
    """r = y - A_S s_S and 1/2||r||^2 per signal.  S, Sv: (B, t); Y: (m, B).
    Returns (R (m, B) column-major, loss (B,))."""
    torch = _torch()
    A = _colmajor(A, torch.float32)
    Y = _colmajor(Y, torch.float32)
    _require_cuda(A, Y, S, Sv)
    m, n = A.shape
    S = S.to(torch.int32).contiguous()
    Sv = Sv.to(torch.float32).contiguous()
    B, t = S.shape
    R = torch.empty((B, m), dtype=torch.float32, device=A.device).t()
    loss = torch.empty(B, dtype=torch.float32, device=A.device)
    _check(load().clfit_forward(ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), ctypes.c_void_p(S.data_ptr()),
                                ctypes.c_void_p(Sv.data_ptr()), t, t, ctypes.c_void_p(Y.data_ptr()),
                                m if B <= 1 else _ld(Y), B, ctypes.c_void_p(R.data_ptr()), m,
                                ctypes.c_void_p(loss.data_ptr()), _stream_ptr(stream)))
    return R, loss


def clfit_adjoint(A, S, R, stream=None):
    """grad = -A_S^T r per signal; S: (B, t); R: (m, B).  Returns (B, t)."""
    torch = _torch()
    A = _colmajor(A, torch.float32)
    R = _colmajor(R, torch.float32)
    _require_cuda(A, R, S)
    m, n = A.shape
    S = S.to(torch.int32).contiguous()
    B, t = S.shape
    grad = torch.empty((B, t), dtype=torch.float32, device=A.device)
    _check(load().clfit_adjoint(ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), ctypes.c_void_p(S.data_ptr()),
                                t, t, ctypes.c_void_p(R.data_ptr()), m if B <= 1 else _ld(R), B,
                                ctypes.c_void_p(grad.data_ptr()), _stream_ptr(stream)))
    return grad


def clfit_adam_step(A, S, Sv, R, mom, vel, tau, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
                    stream=None):
    """Adjoint fused with one Adam step; updates Sv, mom, vel in place and
    returns the gradient (B, t)."""
    torch = _torch()
    A = _colmajor(A, torch.float32)
    R = _colmajor(R, torch.float32)
    m, n = A.shape
    _require_cuda(A, R, S, Sv, mom, vel)
    S = S.to(torch.int32).contiguous()
    for x in (Sv, mom, vel):
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("Sv, mom, vel must be contiguous float32 (B, t) tensors")
    B, t = S.shape
    grad = torch.empty((B, t), dtype=torch.float32, device=A.device)
    _check(load().clfit_adam_step(ctypes.c_void_p(A.data_ptr()), m, n, _ld(A), ctypes.c_void_p(S.data_ptr()),
                                  ctypes.c_void_p(Sv.data_ptr()), t, t, ctypes.c_void_p(R.data_ptr()),
                                  m if B <= 1 else _ld(R), B, ctypes.c_void_p(mom.data_ptr()),
                                  ctypes.c_void_p(vel.data_ptr()), int(tau), float(lr), float(beta1),
                                  float(beta2), float(eps), ctypes.c_void_p(grad.data_ptr()),
                                  _stream_ptr(stream)))
    return grad
