"""GPU parity of the persistent CLOMP solve (bf16 tensor-core correlation,
Gram-form Adam fit, the whole solve in one kernel) against the FP64 oracle
and against the per-iteration kernels."""
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


def solve(cs, torch, A32, Y32, k, persist=1, fuse=1, **kw):
    m, n = A32.shape
    B = Y32.shape[1]
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = cs.Plan(m, n, max(B, 1), k)
    plan.set_option(cs.OPT_PERSIST, persist)
    plan.set_option(cs.OPT_FUSE_UPDATE, fuse)
    cl = dict(CL)
    cl.update(kw)
    r = cs.clomp_solve_batched(A, Y, k, prec="bf16", form="gram", plan=plan, **cl)
    torch.cuda.synchronize()
    launches = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    fallbacks, errs = plan.counters()
    assert errs == 0, f"device error flags {errs:#x}"
    out = to_numpy(r)
    out["launches"] = launches
    out["fallbacks"] = fallbacks
    return out


def oracle_clomp(A64, Y64, k, tol=0.0, max_iter=None, **kw):
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in kw.items() if q in p})
    return oracle.clomp(A64, Y64, k, tol=tol, max_iter=max_iter, steps=kw.get("steps", CL["steps"]),
                        reset_adam=kw.get("reset_adam", False), th=f32(kw.get("th", 0.0)), **p)


def test_persist_matches_per_iteration_kernels(cs_gpu, torch):
    """Same float32 argmax, fit and residual arithmetic: the persistent solve
    reproduces the per-iteration fused kernels."""
    p = workloads.random_problem(77, 301, 333, 20, seed=71, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    ps = solve(cs_gpu, torch, A32, Y32, 20, persist=1)
    it = solve(cs_gpu, torch, A32, Y32, 20, persist=0)
    assert ps["launches"]["persist"] == 1 and ps["launches"]["update"] == 0
    assert it["launches"]["persist"] == 0 and it["launches"]["update"] == 20
    assert np.array_equal(ps["support"], it["support"])
    assert np.array_equal(ps["n_iter"], it["n_iter"]) and np.array_equal(ps["status"], it["status"])
    same = np.all(ps["coef"] == it["coef"], axis=1)
    print("bitwise-identical coefficient rows:", int(same.sum()), "of", len(same))
    np.testing.assert_allclose(ps["coef"], it["coef"], rtol=1e-6, atol=1e-7)


def test_persist_batched_workload_every_signal(cs_gpu, torch):
    """n=1024, m=256, 4096 signals, k=32 (one block of 27 signals per SM) --
    the benchmark's headline solve -- every signal against the oracle."""
    p = workloads.config_batched()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, p.k)
    assert g["launches"]["persist"] == 1
    s = compare(g, oracle_clomp(A64, Y64, p.k))
    print(s, "list overflows:", g["fallbacks"])
    assert s["signals"] == p.B
    assert np.all(g["status"] == 0) and np.all(g["n_iter"] == 32)


@pytest.mark.parametrize("B", [1, 5, 152 * 30 + 7])
def test_persist_ragged_blocks(cs_gpu, torch, B):
    """Batches smaller than the SM count, and larger than one block of 27
    signals per SM (CTAs then run several blocks)."""
    p = workloads.random_problem(77, 301, B, 12, seed=72 + B, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 12)
    idx = np.arange(B) if B <= 64 else np.sort(np.random.default_rng(1).choice(B, 64, replace=False))
    compare(g, oracle_clomp(A64, Y64[:, idx], 12), idx=idx)


@pytest.mark.parametrize("sr", [0.1, 0.5])
def test_persist_columnwise_2d(cs_gpu, torch, sr):
    """Sr = 0.1 (k = 8) runs the persistent solve; Sr = 0.5 (k = 42, above
    its k <= 32) falls back to the per-iteration kernels with the fused
    update, one launch of each per iteration.  Both match the oracle."""
    p = workloads.config_columnwise_2d(sr, n_images=4)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, p.k)
    if p.k <= 32:
        assert g["launches"]["persist"] == 1
    else:
        assert g["launches"]["persist"] == 0 and g["launches"]["update"] == p.k
    idx = np.arange(0, p.B, 8)
    compare(g, oracle_clomp(A64, Y64[:, idx], p.k), idx=idx)


def test_persist_edge_cases(cs_gpu, torch):
    rng = np.random.default_rng(73)
    A = workloads.gaussian_matrix(rng, 16, 40)
    Y = rng.standard_normal((16, 6))
    Y[3, 1] = np.nan          # non-finite -> status 4, no iteration
    Y[:, 2] = 0.0             # ||y|| <= tol before any iteration -> status 1
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = solve(cs_gpu, torch, A32, Y32, 5, tol=1e-6, max_iter=3)
    assert g["status"].tolist() == [2, 4, 1, 2, 2, 2]
    assert g["n_iter"].tolist() == [3, 0, 0, 3, 3, 3]
    assert np.all(g["support"][1] == -1) and np.isnan(g["res_norm"][1])
    o = oracle_clomp(A64, Y64, 5, tol=1e-6, max_iter=3)
    ok = [0, 3, 4, 5]
    compare({q: v[ok] for q, v in g.items() if q in o}, {q: v[ok] for q, v in o.items()})
    # k = 1 and a tolerance stop
    g1 = solve(cs_gpu, torch, A32, Y32[:, [0]], 1)
    compare(g1, oracle_clomp(A64, Y64[:, [0]], 1))


def test_persist_reset_adam_and_graph_replay(cs_gpu, torch):
    p = workloads.random_problem(40, 120, 50, 6, seed=74, snr_db=40.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 6, reset_adam=True, steps=30, lr=2e-2)
    compare(g, oracle_clomp(A64, Y64, 6, reset_adam=True, steps=30, lr=2e-2))
    # eager, captured and replayed solves on one plan agree bit for bit
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(40, 120, 50, 6)
    got = []
    for _ in range(3):
        r = cs_gpu.clomp_solve_batched(A, Y, 6, prec="bf16", plan=plan, **CL)
        torch.cuda.synchronize()
        got.append(to_numpy(r))
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(got[0][q], got[1][q]) and np.array_equal(got[0][q], got[2][q]), q


def test_persist_bounded_wait_reports_timeout(cs_gpu, torch):
    """Failure path of the persistent solve without a GPU fault: the test hook
    withholds one MMA completion signal, the signal warps' bounded wait runs
    out, the kernel shuts down cleanly and the plan reports a device error
    (CS_ETIMEOUT); the next solve on the same plan is correct."""
    p = workloads.random_problem(64, 300, 40, 8, seed=76, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs_gpu.Plan(64, 300, 40, 8)
    plan.set_option(cs_gpu.OPT_STALL_TEST, 1)
    cs_gpu.clomp_solve_batched(A, Y, 8, prec="bf16", plan=plan, **CL)
    torch.cuda.synchronize()                   # returns: every wait is bounded
    _, errs = plan.counters(reset=True)
    # whichever bounded wait runs out first reports: the signal warps' (16)
    # or the MMA issuer's wait for the residuals of the next pass (8)
    assert errs & (8 | 16), f"expected a bounded-wait flag, got {errs:#x}"
    r = cs_gpu.clomp_solve_batched(A, Y, 8, prec="bf16", plan=plan, **CL)
    torch.cuda.synchronize()
    assert plan.counters(reset=True)[1] == 0
    compare(to_numpy(r), oracle_clomp(A64, Y64, 8))


@pytest.mark.parametrize("m,n", [(256, 2048), (250, 2000)])
def test_persist_largest_sizes(cs_gpu, torch, m, n):
    """The persistent solve's limits: n = 2048 atoms (16 atom tiles, the
    key's 11 index bits), m = 256 (four K blocks), k = 32; and a ragged
    neighbour (m = 250 padded to 256, a partial last atom tile)."""
    p = workloads.random_problem(m, n, 300, 32, seed=78 + n, snr_db=40.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = solve(cs_gpu, torch, A32, Y32, 32)
    assert g["launches"]["persist"] == 1
    idx = np.sort(np.random.default_rng(5).choice(300, size=48, replace=False))
    print(compare(g, oracle_clomp(A64, Y64[:, idx], 32), idx=idx), "list overflows:", g["fallbacks"])
