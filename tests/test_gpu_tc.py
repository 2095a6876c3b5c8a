"""GPU checks of the correlation layer C = A^T R (tcgen05 bf16 and float32
SIMT) and of the bf16-correlation solvers against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads
from parity import compare, f32, f32_problem, to_numpy

pytestmark = pytest.mark.gpu

CL = dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _bf16_round(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("m,n,B", [(256, 1024, 333), (26, 300, 129), (77, 40, 1), (128, 513, 200),
                                   (200, 257, 130)])
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_correlate_dense(cs_gpu, torch, m, n, B, prec):
    rng = np.random.default_rng(m * 7 + n + B)
    A = np.asfortranarray(rng.standard_normal((m, n)).astype(np.float32))
    R = np.asfortranarray(rng.standard_normal((m, B)).astype(np.float32))
    C = cs_gpu.correlate(torch.from_numpy(A).cuda(), torch.from_numpy(R).cuda(), prec=prec)
    torch.cuda.synchronize()
    C = C.cpu().numpy().astype(np.float64)
    if prec == "bf16":
        Ar, Rr = _bf16_round(torch, A), _bf16_round(torch, R)
    else:
        Ar, Rr = A.astype(np.float64), R.astype(np.float64)
    ref = Ar.T @ Rr
    bound = (np.abs(Ar).T @ np.abs(Rr)) * (m * 2.0 ** -23) + 1e-30
    err = np.abs(C - ref)
    assert np.all(err <= bound), f"max err {err.max():.3e}, worst ratio {(err / bound).max():.2f}"
    if prec == "bf16":
        # and the bf16 result stays within the certificate's rounding bound of the fp32 truth
        exact = A.astype(np.float64).T @ R.astype(np.float64)
        db = (2.0 ** -7 + 2.0 ** -16 + m * (2.0 ** -22 + 2.0 ** -23)) * \
            np.linalg.norm(A, axis=0)[:, None] * np.linalg.norm(R, axis=0)[None, :]
        assert np.all(np.abs(C - exact) <= db)


@pytest.mark.parametrize("algo,form", [("omp", None), ("clomp", "gram"), ("clomp", "gather")])
def test_bf16_solvers_ragged(cs_gpu, torch, algo, form):
    p = workloads.random_problem(77, 301, 333, 12, seed=41, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(77, 301, 333, 12)
    if algo == "omp":
        r = cs_gpu.omp_solve_batched(A, Y, p.k, prec="bf16", plan=plan)
        o = oracle.omp(A64, Y64, p.k)
    else:
        r = cs_gpu.clomp_solve_batched(A, Y, p.k, prec="bf16", form=form, plan=plan, **CL)
        o = oracle.clomp(A64, Y64, p.k, steps=50, lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999),
                         eps=f32(1e-8))
    fallbacks, errs = plan.counters(reset=True)
    assert errs == 0
    s = compare(to_numpy(r), o)
    print(algo, form, s, "fallbacks", fallbacks)


@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_bf16_batched_workload_sampled(cs_gpu, torch, algo):
    p = workloads.config_batched()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(p.m, p.n, p.B, p.k)
    if algo == "omp":
        r = cs_gpu.omp_solve_batched(A, Y, p.k, prec="bf16", plan=plan)
    else:
        r = cs_gpu.clomp_solve_batched(A, Y, p.k, prec="bf16", form="gram", plan=plan, **CL)
    fallbacks, errs = plan.counters(reset=True)
    assert errs == 0
    g = to_numpy(r)
    idx = np.random.default_rng(1).choice(p.B, size=384, replace=False)
    idx.sort()
    if algo == "omp":
        o = oracle.omp(A64, Y64[:, idx], p.k)
    else:
        o = oracle.clomp(A64, Y64[:, idx], p.k, steps=50, lr=f32(1e-2), beta1=f32(0.9),
                         beta2=f32(0.999), eps=f32(1e-8))
    s = compare(g, o, idx=idx)
    print(algo, s, "fallbacks", fallbacks, "of", p.B * p.k, "picks")


@pytest.mark.parametrize("sr", [0.1, 0.5])
def test_bf16_columnwise_2d_sampled(cs_gpu, torch, sr):
    p = workloads.config_columnwise_2d(sr, n_images=8)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(p.m, p.n, p.B, p.k)
    r = cs_gpu.clomp_solve_batched(A, Y, p.k, prec="bf16", form="gram", plan=plan, **CL)
    fallbacks, errs = plan.counters(reset=True)
    assert errs == 0
    idx = np.arange(0, p.B, 8)
    o = oracle.clomp(A64, Y64[:, idx], p.k, steps=50, lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999),
                     eps=f32(1e-8))
    s = compare(to_numpy(r), o, idx=idx)
    print(sr, s, "fallbacks", fallbacks)


def test_bf16_matches_fp32_selection_bitwise_when_certified(cs_gpu, torch):
    """The bf16 path's float32 re-score makes it pick exactly the float32
    path's atoms; the coefficients then agree bit for bit (same fit kernels)."""
    p = workloads.random_problem(128, 512, 256, 16, seed=42, snr_db=40.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    a = to_numpy(cs_gpu.clomp_solve_batched(A, Y, 16, prec="bf16", **CL))
    b = to_numpy(cs_gpu.clomp_solve_batched(A, Y, 16, prec="fp32", **CL))
    same = np.all(a["support"] == b["support"], axis=1)
    assert same.mean() >= 0.99
    assert np.array_equal(a["coef"][same], b["coef"][same])
