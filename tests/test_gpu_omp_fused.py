"""The fused small-batch OMP solve (one CTA per signal, one launch) gives the
same bits as the per-iteration kernels, and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads
from parity import compare, f32_problem, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def omp(cs, torch, A32, Y32, k, fused, **kw):
    m, n = A32.shape
    B = Y32.shape[1]
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = cs.Plan(m, n, max(B, 1), k)
    plan.set_option(cs.OPT_FUSED_OMP, fused)
    r = cs.omp_solve_batched(A, Y, k, prec="fp32", plan=plan, **kw)
    torch.cuda.synchronize()
    out = to_numpy(r)
    out["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    return out


@pytest.mark.parametrize("m,n,B,k", [(77, 301, 1, 12), (77, 301, 7, 12), (256, 1024, 152, 32),
                                     (700, 900, 20, 30)])
def test_fused_omp_is_bitwise_the_per_iteration_solve(cs_gpu, torch, m, n, B, k):
    p = workloads.random_problem(m, n, B, k, seed=130 + B, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    f = omp(cs_gpu, torch, A32, Y32, k, 1)
    g = omp(cs_gpu, torch, A32, Y32, k, 0)
    assert f["launches"]["persist"] == 1 and f["launches"]["correlation"] == 0
    assert g["launches"]["persist"] == 0 and g["launches"]["correlation"] == k
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(f[q], g[q]), q
    idx = np.arange(B) if B <= 32 else np.arange(0, B, 5)
    compare(f, oracle.omp(A64, Y64[:, idx], k), idx=idx)


def test_fused_omp_single_signal_and_stops(cs_gpu, torch):
    """The single-signal workload (n = 256, m = 64, k = 8, noiseless, tol
    1e-10): recovered exactly; tolerance and max_iter stops, a zero signal."""
    p = workloads.config_single_fp64()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    f = omp(cs_gpu, torch, A32, Y32, p.k, 1, tol=p.tol)
    o = oracle.omp(A64, Y64, p.k, tol=p.tol)
    compare(f, o)
    Y2 = np.concatenate([Y32, np.zeros_like(Y32)], axis=1)
    f2 = omp(cs_gpu, torch, A32, np.asfortranarray(Y2), p.k, 1, tol=p.tol, max_iter=3)
    assert f2["n_iter"].tolist() == [3, 0] and f2["status"].tolist() == [2, 1]


def test_fused_omp_only_for_small_batches(cs_gpu, torch):
    p = workloads.random_problem(64, 200, 400, 6, seed=131, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    f = omp(cs_gpu, torch, A32, Y32, 6, 1)
    assert f["launches"]["persist"] == 0 and f["launches"]["correlation"] == 6


def test_fused_omp_self_contained_reads_callers_layout(cs_gpu, torch):
    """With A resident in shared memory the fused solve is the only launch:
    it reads the caller's A and Y through their leading dimensions (both
    larger than m here) and does the set-up itself -- a NaN signal (status
    4), a zero signal under tol (1) -- with the per-iteration kernels' bits."""
    m, n, B, k = 61, 250, 5, 9
    p = workloads.random_problem(m, n, B, k, seed=133, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    Y32 = np.array(Y32)
    Y32[7, 1] = np.nan
    Y32[:, 3] = 0.0
    Abig = torch.zeros((m + 7, n), dtype=torch.float32).t().contiguous().t().cuda()   # column-major, lda = m + 7
    Abig[:m] = torch.from_numpy(A32).cuda()
    Ybig = torch.zeros((m + 3, B), dtype=torch.float32).t().contiguous().t().cuda()
    Ybig[:m] = torch.from_numpy(Y32).cuda()
    outs = {}
    for fused in (1, 0):
        plan = cs_gpu.Plan(m, n, B, k)
        plan.set_option(cs_gpu.OPT_FUSED_OMP, fused)
        r = cs_gpu.omp_solve_batched(Abig[:m], Ybig[:m], k, prec="fp32", plan=plan, tol=1e-6)
        torch.cuda.synchronize()
        outs[fused] = to_numpy(r)
        outs[fused]["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    f, g = outs[1], outs[0]
    assert sum(f["launches"].values()) == 1 and f["launches"]["persist"] == 1, f["launches"]
    assert f["status"][1] == 4 and f["status"][3] == 1 and f["n_iter"][3] == 0
    for q in ("support", "coef", "n_iter", "status"):
        assert np.array_equal(f[q], g[q]), q
    assert np.array_equal(f["res_norm"], g["res_norm"], equal_nan=True)
    ok = [0, 2, 4]
    compare({q: v[ok] for q, v in f.items() if q != "launches"}, oracle.omp(A64, Y64[:, ok], k, tol=1e-6))
