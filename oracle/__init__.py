"""FP64 CPU oracle for OMP / CLOMP (test infrastructure, not the product).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It compiles ``cs_oracle.c`` with gcc on first
use (or via :func:`build`) and wraps it with ctypes.  It imports nothing from
the GPU package and the GPU package imports nothing from here.

Every function returns float64 results; per-iteration arrays come back as
(B, k) numpy arrays (row b = signal b, in selection order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcs_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off keeps the arithmetic identical on x86-64 and aarch64 hosts
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            d, i32 = ctypes.c_double, ctypes.c_int32
            pd, pi = P(d), P(i32)
            L.cs_oracle_lstsq.argtypes = [ctypes.c_int, ctypes.c_int, pd, ctypes.c_int, pd, pd, pd]
            L.cs_oracle_lstsq.restype = ctypes.c_int
            L.cs_oracle_clfit_loss_grad.argtypes = [pd, ctypes.c_int, ctypes.c_int, pi, ctypes.c_int,
                                                    pd, pd, pd, pd, pd]
            L.cs_oracle_clfit_loss_grad.restype = None
            L.cs_oracle_clfit_adam.argtypes = [pd, ctypes.c_int, ctypes.c_int, pi, ctypes.c_int, pd,
                                               pd, pd, pd, pi, ctypes.c_int, d, d, d, d]
            L.cs_oracle_clfit_adam.restype = None
            L.cs_oracle_omp.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, d, ctypes.c_int, pi, pd, pi, pd, pi,
                                        pd, pd, pd, ctypes.c_int]
            L.cs_oracle_omp.restype = ctypes.c_int
            L.cs_oracle_omp_method.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, d, ctypes.c_int, ctypes.c_int, pi,
                                               pd, pi, pd, pi, pd, pd, pd, ctypes.c_int]
            L.cs_oracle_omp_method.restype = ctypes.c_int
            L.cs_oracle_clomp.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, d, ctypes.c_int, ctypes.c_int, d, d,
                                          d, d, ctypes.c_int, d, d, pd, ctypes.c_int, ctypes.c_int,
                                          pi, pd, pi, pd, pi, pd, pd, pd, ctypes.c_int]
            L.cs_oracle_clomp.restype = ctypes.c_int
            L.cs_oracle_tv_loss_grad.argtypes = [pd, ctypes.c_int, ctypes.c_int, pi, ctypes.c_int, pd, d, pd]
            L.cs_oracle_tv_loss_grad.restype = d
            L.cs_oracle_clomp_image.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, d,
                                                ctypes.c_int, ctypes.c_int, d, d, d, d, ctypes.c_int, d, d, d,
                                                pd, ctypes.c_int, ctypes.c_int, pi, pd, pi, pd, pi, pd,
                                                pd, pd, ctypes.c_int]
            L.cs_oracle_clomp_image.restype = ctypes.c_int
            L.cs_oracle_lv_loss_grad.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, pi, pi, pd, d, d, pd]
            L.cs_oracle_lv_loss_grad.restype = d
            L.cs_oracle_tv2d_h_loss_grad.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, pi, pi, pd, d, pd]
            L.cs_oracle_tv2d_h_loss_grad.restype = d
            L.cs_oracle_iht.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, d, d, ctypes.c_int, pi, pd, pi, pd, pi, pd,
                                        ctypes.c_int]
            L.cs_oracle_iht.restype = ctypes.c_int
            L.cs_oracle_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64F(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(lib().cs_oracle_max_threads())


def lstsq(As, y):
    """min ||y - As z|| by Householder QR.  Returns (z, status) with status 3
    when the last column is dependent."""
    As = _f64F(As)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m, t = As.shape
    z = np.zeros(t)
    work = np.zeros(m * t + m)
    st = lib().cs_oracle_lstsq(m, t, _p(As, ctypes.c_double), m, _p(y, ctypes.c_double),
                               _p(z, ctypes.c_double), _p(work, ctypes.c_double))
    return z, st


def clfit_loss_grad(A, support, s_S, y):
    """L = 1/2||y - A_S s_S||^2 and its gradient -(A_S^T r); returns (L, grad, r)."""
    A = _f64F(A)
    S = np.ascontiguousarray(support, dtype=np.int32)
    s = np.ascontiguousarray(s_S, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m = A.shape[0]
    loss = np.zeros(1)
    g = np.zeros(len(S))
    r = np.zeros(m)
    lib().cs_oracle_clfit_loss_grad(_p(A, ctypes.c_double), m, m, _p(S, ctypes.c_int32), len(S),
                                    _p(s, ctypes.c_double), _p(y, ctypes.c_double),
                                    _p(loss, ctypes.c_double), _p(g, ctypes.c_double),
                                    _p(r, ctypes.c_double))
    return float(loss[0]), g, r


def clfit_adam(A, support, y, s_S, mom, vel, tau, steps, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """Run `steps` Adam steps of the CL fit in place-free form; returns
    (s_S, mom, vel, tau)."""
    A = _f64F(A)
    S = np.ascontiguousarray(support, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.float64)
    s = np.array(s_S, dtype=np.float64)
    mo = np.array(mom, dtype=np.float64)
    ve = np.array(vel, dtype=np.float64)
    ta = np.array([tau], dtype=np.int32)
    m = A.shape[0]
    lib().cs_oracle_clfit_adam(_p(A, ctypes.c_double), m, m, _p(S, ctypes.c_int32), len(S),
                               _p(y, ctypes.c_double), _p(s, ctypes.c_double),
                               _p(mo, ctypes.c_double), _p(ve, ctypes.c_double),
                               _p(ta, ctypes.c_int32), int(steps), lr, beta1, beta2, eps)
    return s, mo, ve, int(ta[0])


def _outputs(B, k):
    return dict(support=np.zeros((B, k), np.int32), coef=np.zeros((B, k)),
                n_iter=np.zeros(B, np.int32), res_norm=np.zeros(B), status=np.zeros(B, np.int32),
                top1=np.zeros((B, k)), top2=np.zeros((B, k)), res_hist=np.zeros((B, k)))


_OMP_METHODS = {"auto": 0, "householder": 1, "iqr": 2}


def omp(A, Y, k, tol=0.0, max_iter=None, nthreads=0, method="auto"):
    """Plain OMP for every column of Y.  Returns a dict of outputs.
    method: "householder" refactorises A_S by Householder QR every
    iteration, "iqr" grows a QR factorisation by modified Gram-Schmidt
    (twice) one column per iteration, "auto" takes the latter when the
    refactorisations would cost m k^3 / 3 > 1e9 flops.  A single signal correlates with the atoms split over the
    threads."""
    A = _f64F(A)
    Y = _f64F(Y if np.ndim(Y) == 2 else np.reshape(Y, (-1, 1)))
    m, n = A.shape
    B = Y.shape[1]
    max_iter = k if max_iter is None else max_iter
    o = _outputs(B, k)
    rc = lib().cs_oracle_omp_method(_p(A, ctypes.c_double), m, n, m, _p(Y, ctypes.c_double), m, B, k,
                             float(tol), int(max_iter), _OMP_METHODS[method], _p(o["support"], ctypes.c_int32),
                             _p(o["coef"], ctypes.c_double), _p(o["n_iter"], ctypes.c_int32),
                             _p(o["res_norm"], ctypes.c_double), _p(o["status"], ctypes.c_int32),
                             _p(o["top1"], ctypes.c_double), _p(o["top2"], ctypes.c_double),
                             _p(o["res_hist"], ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError("cs_oracle_omp: invalid arguments")
    return o


def iht(A, Y, k, step, tol=0.0, max_iter=200, nthreads=0):
    """IHT for every column of Y: s <- H_k(s + step A^T r), at most max_iter
    iterations.  Returns support (ascending), coef, n_iter, res_norm, status
    and margin (the smallest relative gap at the k-th largest |u|)."""
    A = _f64F(A)
    Y = _f64F(Y if np.ndim(Y) == 2 else np.reshape(Y, (-1, 1)))
    m, n = A.shape
    B = Y.shape[1]
    o = dict(support=np.zeros((B, k), np.int32), coef=np.zeros((B, k)), n_iter=np.zeros(B, np.int32),
             res_norm=np.zeros(B), status=np.zeros(B, np.int32), margin=np.zeros(B))
    rc = lib().cs_oracle_iht(_p(A, ctypes.c_double), m, n, m, _p(Y, ctypes.c_double), m, B, int(k), float(step),
                             float(tol), int(max_iter), _p(o["support"], ctypes.c_int32),
                             _p(o["coef"], ctypes.c_double), _p(o["n_iter"], ctypes.c_int32),
                             _p(o["res_norm"], ctypes.c_double), _p(o["status"], ctypes.c_int32),
                             _p(o["margin"], ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError("cs_oracle_iht: invalid arguments")
    return o


def tv_loss_grad(D, n, support, s_S, w):
    """w * TV(x) of Eq. 5 for x = D[:, support] @ s_S (D None: x = s placed
    at `support` in a length-n vector) and its gradient w.r.t. s_S."""
    S = np.ascontiguousarray(support, dtype=np.int32)
    s_S = np.ascontiguousarray(s_S, dtype=np.float64)
    g = np.zeros(len(S))
    if D is None:
        val = lib().cs_oracle_tv_loss_grad(None, int(n), int(n), _p(S, ctypes.c_int32), len(S),
                                           _p(s_S, ctypes.c_double), float(w), _p(g, ctypes.c_double))
    else:
        Df = _f64F(D)
        val = lib().cs_oracle_tv_loss_grad(_p(Df, ctypes.c_double), Df.shape[0], Df.shape[0],
                                           _p(S, ctypes.c_int32), len(S), _p(s_S, ctypes.c_double),
                                           float(w), _p(g, ctypes.c_double))
    return val, g


def _image_loss_grad(fn, D, n, supports, coefs, w, *extra):
    W = len(supports)
    k = max(1, max(len(q) for q in supports))
    S = np.full((W, k), -1, np.int32)
    C = np.zeros((W, k))
    t = np.zeros(W, np.int32)
    for j, (sj, cj) in enumerate(zip(supports, coefs)):
        t[j] = len(sj)
        S[j, :len(sj)] = sj
        C[j, :len(sj)] = cj
    G = np.zeros((W, k))
    if D is None:
        Dp, N = None, int(n)
    else:
        Df = _f64F(D)
        Dp, N = _p(Df, ctypes.c_double), Df.shape[0]
    val = fn(Dp, N, N, W, k, _p(S, ctypes.c_int32), _p(t, ctypes.c_int32), _p(C, ctypes.c_double),
             float(w), *[float(e) for e in extra], _p(G, ctypes.c_double))
    return val, [G[j, :t[j]].copy() for j in range(W)]


def tv2d_h_loss_grad(D, n, supports, coefs, w):
    """w * TV_h(I), the horizontal part of Eq. 6, for the image whose column j
    is x_j = D[:, supports[j]] @ coefs[j] (D None: x_j = coefs[j] placed at
    supports[j] in a length-n vector), and its gradient: a list of arrays,
    one per column, w.r.t. coefs[j]."""
    return _image_loss_grad(lib().cs_oracle_tv2d_h_loss_grad, D, n, supports, coefs, w)


def lv_loss_grad(D, n, supports, coefs, w, eps=0.0):
    """w * LV(I) of Eq. 7 (3 x 3 windows at every placement, sample standard
    deviation smoothed as sqrt(var + eps^2)) for the image of columns x_j as
    in tv2d_h_loss_grad, and its gradient w.r.t. coefs[j]."""
    return _image_loss_grad(lib().cs_oracle_lv_loss_grad, D, n, supports, coefs, w, eps)


def clomp(A, Y, k, tol=0.0, max_iter=None, steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
          reset_adam=False, th=0.0, tv_weight=0.0, D=None, image_width=0, lv_weight=0.0, lv_eps=0.0,
          nthreads=0):
    """CLOMP (structure 1, Adam) for every column of Y.  Returns a dict.

    th: 0 selects one atom per iteration (argmax); 0 < th < 1 selects every
    unselected atom with |c| >= th * max|c| per iteration (largest first, at
    most k in total); n_iter then counts atoms.  top1/top2 of such picks hold
    1 and 1 - margin, margin being the smallest relative gap deciding the
    iteration's set and order.  tv_weight > 0 adds tv_weight * TV(D s) (Eq. 5)
    to the fit's loss; D (N x n) None means x = s.  image_width = W >= 1 reads
    the batch as images of W consecutive columns and uses the image form of
    the prior (Eq. 6), which couples neighbouring columns in the fit;
    lv_weight > 0 (with image_width) adds lv_weight * LV(I) of Eq. 7, each
    window's deviation smoothed as sqrt(var + lv_eps^2)."""
    A = _f64F(A)
    Y = _f64F(Y if np.ndim(Y) == 2 else np.reshape(Y, (-1, 1)))
    m, n = A.shape
    B = Y.shape[1]
    max_iter = k if max_iter is None else max_iter
    o = _outputs(B, k)
    Df = None if D is None else _f64F(D)
    Dp = None if Df is None else _p(Df, ctypes.c_double)
    N = n if Df is None else Df.shape[0]
    if lv_weight and not image_width:
        raise ValueError("the local variation needs image_width")
    if image_width:
        if th:
            raise ValueError("the image prior runs with one atom per iteration (th = 0)")
        rc = lib().cs_oracle_clomp_image(_p(A, ctypes.c_double), m, n, m, _p(Y, ctypes.c_double), m, B,
                                        int(image_width), k, float(tol), int(max_iter), int(steps), float(lr),
                                        float(beta1), float(beta2), float(eps), int(bool(reset_adam)),
                                        float(tv_weight), float(lv_weight), float(lv_eps), Dp, int(N), int(N),
                                        _p(o["support"], ctypes.c_int32), _p(o["coef"], ctypes.c_double),
                                        _p(o["n_iter"], ctypes.c_int32), _p(o["res_norm"], ctypes.c_double),
                                        _p(o["status"], ctypes.c_int32), _p(o["top1"], ctypes.c_double),
                                        _p(o["top2"], ctypes.c_double), _p(o["res_hist"], ctypes.c_double),
                                        int(nthreads))
        if rc != 0:
            raise ValueError("cs_oracle_clomp_image: invalid arguments")
        return o
    rc = lib().cs_oracle_clomp(_p(A, ctypes.c_double), m, n, m, _p(Y, ctypes.c_double), m, B, k,
                               float(tol), int(max_iter), int(steps), float(lr), float(beta1),
                               float(beta2), float(eps), int(bool(reset_adam)), float(th),
                               float(tv_weight), Dp, int(N), int(N),
                               _p(o["support"], ctypes.c_int32), _p(o["coef"], ctypes.c_double),
                               _p(o["n_iter"], ctypes.c_int32), _p(o["res_norm"], ctypes.c_double),
                               _p(o["status"], ctypes.c_int32), _p(o["top1"], ctypes.c_double),
                               _p(o["top2"], ctypes.c_double), _p(o["res_hist"], ctypes.c_double),
                               int(nthreads))
    if rc != 0:
        raise ValueError("cs_oracle_clomp: invalid arguments")
    return o
