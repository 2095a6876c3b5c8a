"""GPU parity of the total-variation prior of Eq. 5 in the CL fit (x = D s,
loss 1/2||y - A_S s_S||^2 + w TV(x)) against the FP64 oracle."""
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


def gpu_solve(cs, torch, A32, Y32, k, prec="bf16", persist=1, D32=None, **kw):
    m, n = A32.shape
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    D = None if D32 is None else torch.from_numpy(np.asfortranarray(D32)).cuda()
    plan = cs.Plan(m, n, max(Y32.shape[1], 1), k)
    plan.set_option(cs.OPT_PERSIST, persist)
    cl = dict(CL)
    cl.update(kw)
    r = cs.clomp_solve_batched(A, Y, k, prec=prec, form="gram", plan=plan, D=D, **cl)
    torch.cuda.synchronize()
    assert plan.counters()[1] == 0
    out = to_numpy(r)
    out["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    return out


def oracle_tv(A64, Y64, k, w, D64=None, **kw):
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in kw.items() if q in p})
    return oracle.clomp(A64, Y64, k, steps=kw.get("steps", CL["steps"]), tv_weight=f32(w), D=D64,
                        th=f32(kw.get("th", 0.0)), **p)


@pytest.mark.parametrize("prec,persist", [("bf16", 1), ("bf16", 0), ("fp32", 0)])
def test_tv_prior_without_basis(cs_gpu, torch, prec, persist):
    """x = s: the prior penalises differences of neighbouring coefficients."""
    p = workloads.random_problem(64, 200, 120, 8, seed=120, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = gpu_solve(cs_gpu, torch, A32, Y32, 8, prec=prec, persist=persist, tv_weight=0.5)
    assert (g["launches"]["persist"] == 1) == (prec == "bf16" and persist == 1)
    print(compare(g, oracle_tv(A64, Y64, 8, 0.5)))


def test_tv_prior_columnwise_dct_basis(cs_gpu, torch):
    """The column-wise image workload (A = Phi D, D the orthonormal DCT): the
    prior acts on each image column x = D s."""
    p = workloads.config_columnwise_2d(0.3, n_images=1)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    D = p.meta["D"]
    D32 = np.asfortranarray(D, dtype=np.float32)
    w = 2.0
    g = gpu_solve(cs_gpu, torch, A32, Y32, p.k, D32=D32, tv_weight=w)
    idx = np.arange(0, 256, 2)
    s = compare(g, oracle_tv(A64, Y64[:, idx], p.k, w, D64=D32.astype(np.float64)), idx=idx)
    g0 = gpu_solve(cs_gpu, torch, A32, Y32, p.k)
    print(s, "coefficients moved by the prior (mean |diff|):", np.abs(g["coef"] - g0["coef"]).mean())
    assert np.abs(g["coef"] - g0["coef"]).max() > 0.0


def test_tv_prior_with_threshold_rule(cs_gpu, torch):
    p = workloads.random_problem(64, 200, 60, 10, seed=121, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = gpu_solve(cs_gpu, torch, A32, Y32, 10, prec="fp32", tv_weight=0.3, th=0.7)
    compare(g, oracle_tv(A64, Y64, 10, 0.3, th=0.7))


def test_tv_prior_zero_weight_and_limits(cs_gpu, torch):
    p = workloads.random_problem(40, 120, 30, 6, seed=122, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    D32 = np.asfortranarray(workloads.dct_synthesis(120), dtype=np.float32)
    a = gpu_solve(cs_gpu, torch, A32, Y32, 6, D32=D32, tv_weight=0.0)
    b = gpu_solve(cs_gpu, torch, A32, Y32, 6)
    for q in ("support", "coef", "n_iter", "status"):
        assert np.array_equal(a[q], b[q]), q
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 6, prec="bf16", form="gather", tv_weight=0.5)
    assert e.value.code == cs_gpu.CS_ENOTSUP
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 6, prec="bf16", tv_weight=-1.0)
    assert e.value.code == cs_gpu.CS_EINVAL
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 6, prec="bf16", tv_weight=0.5, D=torch.ones((1, 120), device="cuda"))
    assert e.value.code == cs_gpu.CS_EINVAL
