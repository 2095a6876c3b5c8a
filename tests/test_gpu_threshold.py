"""GPU parity of the threshold selection rule (Th, Methods: every unselected
atom with |c_j| >= Th * max|c| joins the support in the iteration, largest
first, until k atoms) against the FP64 oracle.  The rule runs with the
float32 correlation and the Gram-form CLOMP fit."""
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


def solve(cs, torch, A32, Y32, k, th, plan=None, **kw):
    m, n = A32.shape
    B = Y32.shape[1]
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = plan or cs.Plan(m, n, max(B, 1), k)
    cl = dict(CL)
    cl.update(kw)
    r = cs.clomp_solve_batched(A, Y, k, prec="fp32", form="gram", plan=plan, th=th, **cl)
    torch.cuda.synchronize()
    launches = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    _, errs = plan.counters()
    assert errs == 0, f"device error flags {errs:#x}"
    out = to_numpy(r)
    out["launches"] = launches
    return out


def oracle_th(A64, Y64, k, th, tol=0.0, max_iter=None, **kw):
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in kw.items() if q in p})
    return oracle.clomp(A64, Y64, k, tol=tol, max_iter=max_iter, steps=kw.get("steps", CL["steps"]),
                        reset_adam=kw.get("reset_adam", False), th=f32(th), **p)


@pytest.mark.parametrize("th", [0.7, 0.9])
def test_threshold_batched_sampled(cs_gpu, torch, th):
    """The benchmark's signal model (n=1024, m=256, k=32, +-(1+|N|) values,
    40 dB), 768 signals, 96 sampled against the oracle."""
    p = workloads.config_batched(B=768)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, p.k, th)
    iters = g["launches"]["update"]
    assert g["launches"]["correlation"] == iters and 1 <= iters <= p.k
    idx = np.sort(np.random.default_rng(3).choice(p.B, size=96, replace=False))
    s = compare(g, oracle_th(A64, Y64[:, idx], p.k, th), idx=idx)
    print(th, s, "mean support size:", g["n_iter"].mean())
    assert np.all(g["n_iter"] <= p.k)


def test_threshold_full_batch(cs_gpu, torch):
    """All 4096 signals of the benchmark workload in one solve, sampled."""
    p = workloads.config_batched()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, p.k, 0.7)
    idx = np.sort(np.random.default_rng(4).choice(p.B, size=64, replace=False))
    print(compare(g, oracle_th(A64, Y64[:, idx], p.k, 0.7), idx=idx))
    # every support is a set of distinct atoms, -1 padded after n_iter
    for b in range(0, p.B, 97):
        t = int(g["n_iter"][b])
        assert len(set(g["support"][b, :t].tolist())) == t and np.all(g["support"][b, t:] == -1)


def test_threshold_columnwise(cs_gpu, torch):
    p = workloads.config_columnwise_2d(0.3, n_images=2)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, p.k, 0.7, max_iter=8)
    idx = np.arange(0, p.B, 4)
    compare(g, oracle_th(A64, Y64[:, idx], p.k, 0.7, max_iter=8), idx=idx)


@pytest.mark.parametrize("B", [1, 5, 131])
def test_threshold_ragged(cs_gpu, torch, B):
    """Batches that fill no block of four signals, n not a multiple of 32."""
    p = workloads.random_problem(77, 301, B, 12, seed=80 + B, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 12, 0.6)
    compare(g, oracle_th(A64, Y64, 12, 0.6))


def test_threshold_edge_cases(cs_gpu, torch):
    rng = np.random.default_rng(81)
    A = workloads.gaussian_matrix(rng, 16, 40)
    Y = rng.standard_normal((16, 6))
    Y[3, 1] = np.nan          # non-finite -> status 4, no iteration
    Y[:, 2] = 0.0             # ||y|| <= tol before any iteration -> status 1
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = solve(cs_gpu, torch, A32, Y32, 5, 0.5, tol=1e-6, max_iter=1)
    assert g["status"][1] == 4 and g["n_iter"][1] == 0 and np.all(g["support"][1] == -1)
    assert g["status"][2] == 1 and g["n_iter"][2] == 0
    ok = [0, 3, 4, 5]
    o = oracle_th(A64, Y64, 5, 0.5, tol=1e-6, max_iter=1)
    compare({q: v[ok] for q, v in g.items() if q in o}, {q: v[ok] for q, v in o.items()})
    # one iteration may fill the support: k atoms at once
    g1 = solve(cs_gpu, torch, A32, Y32[:, [0, 3]], 3, 0.05, max_iter=1)
    assert np.all(g1["n_iter"] == 3) and np.all(g1["status"] == 0)
    compare(g1, oracle_th(A64, Y64[:, [0, 3]], 3, 0.05, max_iter=1))


def test_threshold_near_one_is_the_argmax_rule(cs_gpu, torch):
    """Th just below 1 admits only atoms tied with the largest: the float32
    argmax solve (per-iteration kernels) gives the same supports."""
    p = workloads.random_problem(64, 256, 200, 8, seed=82, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 8, 1.0 - 2.0 ** -20)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    r = to_numpy(cs_gpu.clomp_solve_batched(A, Y, 8, prec="fp32", form="gram", **CL))
    same = np.all(g["support"] == r["support"], axis=1)
    assert same.mean() >= 0.99, same.mean()
    np.testing.assert_allclose(g["coef"][same], r["coef"][same], rtol=1e-5, atol=1e-6)


def test_threshold_graph_replay_and_reset_adam(cs_gpu, torch):
    p = workloads.random_problem(40, 120, 50, 6, seed=83, snr_db=40.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 6, 0.8, reset_adam=True, steps=30, lr=2e-2)
    compare(g, oracle_th(A64, Y64, 6, 0.8, reset_adam=True, steps=30, lr=2e-2))
    # eager, captured and replayed solves on one plan agree bit for bit
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(40, 120, 50, 6)
    got = []
    for _ in range(3):
        r = cs_gpu.clomp_solve_batched(A, Y, 6, prec="fp32", plan=plan, th=0.8, **CL)
        torch.cuda.synchronize()
        got.append(to_numpy(r))
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(got[0][q], got[1][q]) and np.array_equal(got[0][q], got[2][q]), q


def test_threshold_rule_limits(cs_gpu, torch):
    A = torch.randn(32, 100, device="cuda")
    Y = torch.randn(32, 4, device="cuda")
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 4, prec="bf16", th=0.7)      # bf16 correlation
    assert e.value.code == cs_gpu.CS_ENOTSUP
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 4, prec="fp32", form="gather", th=0.7)
    assert e.value.code == cs_gpu.CS_ENOTSUP
    with pytest.raises(cs_gpu.CSError):
        cs_gpu.clomp_solve_batched(A, Y, 4, prec="fp32", th=-0.5)


@pytest.mark.parametrize("m", [400, 700])
def test_threshold_larger_m(cs_gpu, torch, m):
    """Row chunks beyond two (m > 256: the kernel's 4- and 8-chunk forms)."""
    p = workloads.random_problem(m, 900, 40, 20, seed=84 + m, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 20, 0.7)
    compare(g, oracle_th(A64, Y64, 20, 0.7))
