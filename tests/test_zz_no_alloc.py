"""The allocation-free OMP entry point, called through the C ABI, gives the
same results as the plan-based omp_solve_batched -- on two calls in a row,
since both share one static scratch array -- and refuses problems that do
not fit its fixed scratch.  Collected last on purpose."""
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
    return fn


def _call(cs, fn, A, Y, k, prec):
    import torch
    m, n = A.shape
    B = Y.shape[1]
    o = cs._outputs(B, k, A.device)
    p = cs.OmpParams(k, 0.0, 0, cs.PREC[prec], 0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = fn(ptr(A), m, n, m, ptr(Y), m, B, ptr(o.support), ptr(o.coef), ptr(o.n_iter),
            ptr(o.res_norm), ptr(o.status), ctypes.byref(p),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, o


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_matches_plan_solver_twice(cs_gpu, prec):
    import torch
    fn = _noalloc(cs_gpu)
    probs = [workloads.random_problem(96, 400, 300, 16, seed=51, snr_db=40.0, values="pm"),
             workloads.random_problem(77, 301, 129, 12, seed=52, snr_db=30.0)]
    for p in probs:             # two different calls in a row on the shared scratch
        A = torch.from_numpy(np.asfortranarray(p.A, dtype=np.float32)).cuda()
        Y = torch.from_numpy(np.asfortranarray(p.Y, dtype=np.float32)).cuda()
        rc, got = _call(cs_gpu, fn, A, Y, p.k, prec)
        assert rc == 0, cs_gpu.load().cs_last_error()
        ref = cs_gpu.omp_solve_batched(A, Y, p.k, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(got.support, ref.support)
        assert torch.equal(got.n_iter, ref.n_iter) and torch.equal(got.status, ref.status)
        c, r = got.coef.double().cpu().numpy(), ref.coef.double().cpu().numpy()
        err = np.linalg.norm(c - r, axis=1) / np.linalg.norm(r, axis=1)
        assert err.max() <= COEF_RTOL


def test_noalloc_rejects_problems_beyond_its_scratch(cs_gpu):
    import torch
    fn = _noalloc(cs_gpu)
    A = torch.zeros(256, 1024, device="cuda").t().contiguous().t()
    Y = torch.zeros(256, 8192, device="cuda").t().contiguous().t()
    rc, _ = _call(cs_gpu, fn, A, Y, 32, "fp32")
    assert rc == -1
    assert b"scratch" in cs_gpu.load().cs_last_error()
