"""The allocation-free OMP entry point, called through the C ABI, gives the
same results as the plan-based omp_solve_batched -- on calls in a row of
different shapes, since all share one static scratch array -- reports its
device counters through omp_solve_batched_noalloc_counters, and refuses
problems that do not fit its fixed scratch.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads
from parity import COEF_RTOL

pytestmark = pytest.mark.gpu


def _noalloc(cs):
    L = cs.load()
    fn = L.omp_solve_batched_noalloc
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    fn.argtypes = [vp, i32, i32, i32, vp, i32, i32, vp, vp, vp, vp, vp,
                   ctypes.POINTER(cs.OmpParams), vp]
    fn.restype = ctypes.c_int
    L.omp_solve_batched_noalloc_counters.argtypes = [vp, i32, vp]
    L.omp_solve_batched_noalloc_counters.restype = ctypes.c_int
    return fn


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call(cs, fn, A, Y, k, prec):
    m, n = A.shape
    B = Y.shape[1]
    o = cs._outputs(B, k, A.device)
    p = cs.OmpParams(k, 0.0, 0, cs.PREC[prec], 0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = fn(ptr(A), m, n, m, ptr(Y), m, B, ptr(o.support), ptr(o.coef), ptr(o.n_iter),
            ptr(o.res_norm), ptr(o.status), ctypes.byref(p), _stream())
    return rc, o


def _noalloc_counters(cs):
    out = np.zeros(4, np.uint32)
    rc = cs.load().omp_solve_batched_noalloc_counters(ctypes.c_void_p(out.ctypes.data), 1, _stream())
    return rc, int(out[0]), int(out[1])


def _check_against_plan(cs, fn, p, prec):
    """One no-alloc call against omp_solve_batched on a fresh plan: identical
    supports, iteration counts and status, coefficients within the parity
    tolerance, and the same certificate-fallback count, with no error flag."""
    import torch
    A = torch.from_numpy(np.asfortranarray(p.A, dtype=np.float32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(p.Y, dtype=np.float32)).cuda()
    rc, got = _call(cs, fn, A, Y, p.k, prec)
    assert rc == 0, cs.load().cs_last_error()
    rc, fallbacks, flags = _noalloc_counters(cs)
    assert rc == 0 and flags == 0, cs.load().cs_last_error()
    plan = cs.Plan(A.shape[0], A.shape[1], Y.shape[1], p.k)
    ref = cs.omp_solve_batched(A, Y, p.k, prec=prec, plan=plan)
    ref_fallbacks, ref_flags = plan.counters(reset=True)
    torch.cuda.synchronize()
    assert ref_flags == 0
    assert fallbacks == ref_fallbacks
    assert torch.equal(got.support, ref.support)
    assert torch.equal(got.n_iter, ref.n_iter) and torch.equal(got.status, ref.status)
    c, r = got.coef.double().cpu().numpy(), ref.coef.double().cpu().numpy()
    err = np.linalg.norm(c - r, axis=1) / np.linalg.norm(r, axis=1)
    assert err.max() <= COEF_RTOL


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_matches_plan_solver_twice(cs_gpu, prec):
    fn = _noalloc(cs_gpu)
    probs = [workloads.random_problem(96, 400, 300, 16, seed=51, snr_db=40.0, values="pm"),
             workloads.random_problem(77, 301, 129, 12, seed=52, snr_db=30.0)]
    for p in probs:             # two different calls in a row on the shared scratch
        _check_against_plan(cs_gpu, fn, p, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_large_batch_after_smaller_call(cs_gpu, prec):
    """More signals than SMs (the per-iteration kernels, not the fused
    small-batch solve) at n = 1024, m = 256, k = 32, right after a smaller
    call of another shape has left its data in the array."""
    fn = _noalloc(cs_gpu)
    small = workloads.random_problem(64, 256, 40, 8, seed=53, snr_db=40.0, values="pm")
    large = workloads.random_problem(256, 1024, 1200, 32, seed=54, snr_db=40.0, values="pm")
    _check_against_plan(cs_gpu, fn, small, prec)
    _check_against_plan(cs_gpu, fn, large, prec)
    _check_against_plan(cs_gpu, fn, small, prec)


def test_noalloc_rejects_problems_beyond_its_scratch(cs_gpu):
    import torch
    fn = _noalloc(cs_gpu)
    A = torch.zeros(256, 1024, device="cuda").t().contiguous().t()
    Y = torch.zeros(256, 8192, device="cuda").t().contiguous().t()
    rc, _ = _call(cs_gpu, fn, A, Y, 32, "fp32")
    assert rc == -1
    assert b"scratch" in cs_gpu.load().cs_last_error()
