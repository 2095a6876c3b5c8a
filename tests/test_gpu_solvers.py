"""GPU parity of the batched OMP / CLOMP solvers against the FP64 oracle.

Every test calls the CUDA library through the C ABI (via the ctypes binding)
and compares with the oracle on the same float32-rounded inputs, using the
rules in tests/parity.py.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity import compare, f32, f32_problem, to_numpy

pytestmark = pytest.mark.gpu

CL = dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)


def _dev(torch, x):
    return torch.from_numpy(np.asfortranarray(x)).cuda()


def run_gpu(cs, torch, A32, Y32, k, algo, **kw):
    A = _dev(torch, A32)
    Y = _dev(torch, Y32)
    if algo == "omp":
        r = cs.omp_solve_batched(A, Y, k, **kw)
    else:
        r = cs.clomp_solve_batched(A, Y, k, **kw)
    torch.cuda.synchronize()
    return to_numpy(r)


def run_oracle(A64, Y64, k, algo, tol=0.0, max_iter=None, **cl):
    if algo == "omp":
        return oracle.omp(A64, Y64, k, tol=tol, max_iter=max_iter)
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in cl.items() if q in p})
    return oracle.clomp(A64, Y64, k, tol=tol, max_iter=max_iter,
                        steps=cl.get("steps", CL["steps"]), reset_adam=cl.get("reset_adam", False), **p)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def test_single_signal_omp(cs_gpu, torch):
    p = workloads.config_single_fp64()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = run_gpu(cs_gpu, torch, A32, Y32, p.k, "omp", tol=p.tol)
    o = run_oracle(A64, Y64, p.k, "omp", tol=p.tol)
    # tol = 1e-10 is below float32 resolution: the GPU stops on |S| = k instead
    compare(g, o, status_equiv={(0, 1)})
    truth = np.nonzero(p.X_true[:, 0])[0]
    assert sorted(g["support"][0].tolist()) == sorted(truth.tolist())


@pytest.mark.parametrize("algo,form", [("omp", None), ("clomp", "gram"), ("clomp", "gather")])
def test_ragged_sizes(cs_gpu, torch, algo, form):
    """m, n, batch off every tile multiple; noisy signals."""
    p = workloads.random_problem(77, 301, 333, 12, seed=11, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    kw = {} if algo == "omp" else dict(form=form, **CL)
    g = run_gpu(cs_gpu, torch, A32, Y32, p.k, algo, **kw)
    o = run_oracle(A64, Y64, p.k, algo)
    s = compare(g, o)
    print(algo, form, s)


@pytest.mark.parametrize("m,k", [(600, 30), (600, 40)])
def test_gather_form_long_columns(cs_gpu, torch, m, k):
    """The gather-form fit beyond 256 rows (float32 correlation): four rows
    per thread over 150 threads, support tiles up to 32 and up to 64."""
    p = workloads.random_problem(m, 900, 24, k, seed=13 + k, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = run_gpu(cs_gpu, torch, A32, Y32, p.k, "clomp", prec="fp32", form="gather", **CL)
    print(compare(g, run_oracle(A64, Y64, p.k, "clomp")))


_BATCHED_ORACLE = {}


def batched_oracle(algo):
    """The FP64 oracle over all 4096 signals of the benchmark workload (once
    per algorithm and module)."""
    if algo not in _BATCHED_ORACLE:
        p = workloads.config_batched()
        _, _, A64, Y64 = f32_problem(p.A, p.Y)
        _BATCHED_ORACLE[algo] = run_oracle(A64, Y64, p.k, algo)
    return _BATCHED_ORACLE[algo]


@pytest.mark.parametrize("algo,prec,form", [("omp", "fp32", None), ("omp", "bf16", None),
                                            ("clomp", "fp32", "gram"), ("clomp", "bf16", "gather")])
def test_batched_workload_every_signal(cs_gpu, torch, algo, prec, form):
    """n=1024, m=256, 4096 signals, k=32 -- the benchmark's launch
    configuration -- every signal against the FP64 oracle (plain fp32 OMP,
    bf16 OMP, fp32 CLOMP in Gram form, bf16 CLOMP in the literal gather
    form; the bf16 Gram form is the persistent solve, tested beside it)."""
    p = workloads.config_batched()
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    kw = dict(prec=prec) if algo == "omp" else dict(prec=prec, form=form, **CL)
    g = run_gpu(cs_gpu, torch, A32, Y32, p.k, algo, **kw)
    s = compare(g, batched_oracle(algo))
    print(algo, prec, form, s)
    assert s["signals"] == p.B
    assert np.all(g["status"] == 0) and np.all(g["n_iter"] == 32)


@pytest.mark.parametrize("sr", [0.1, 0.3, 0.5])
@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_columnwise_2d_sampled(cs_gpu, torch, sr, algo):
    p = workloads.config_columnwise_2d(sr, n_images=8)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    kw = {} if algo == "omp" else dict(form="gram", **CL)
    g = run_gpu(cs_gpu, torch, A32, Y32, p.k, algo, **kw)
    idx = np.arange(0, p.B, 8)
    o = run_oracle(A64, Y64[:, idx], p.k, algo)
    s = compare(g, o, idx=idx)
    print(sr, algo, s)


def test_edge_cases(cs_gpu, torch):
    rng = np.random.default_rng(21)
    A = workloads.gaussian_matrix(rng, 16, 40)
    Y = rng.standard_normal((16, 6))
    Y[3, 1] = np.nan          # non-finite -> status 4, no iteration
    Y[:, 2] = 0.0             # ||y|| <= tol before any iteration -> status 1
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = run_gpu(cs_gpu, torch, A32, Y32, 5, "omp", tol=1e-6, max_iter=3)
    o = run_oracle(A64, Y64, 5, "omp", tol=1e-6, max_iter=3)
    assert g["status"].tolist() == [2, 4, 1, 2, 2, 2]
    assert g["n_iter"].tolist() == [3, 0, 0, 3, 3, 3]
    assert np.all(g["support"][1] == -1) and np.isnan(g["res_norm"][1])
    ok = [0, 3, 4, 5]
    compare({q: v[ok] for q, v in g.items()}, {q: v[ok] for q, v in o.items()})
    # k = 1 and k = m (largest sparsity the problem allows)
    for k in (1, 16):
        g = run_gpu(cs_gpu, torch, A32, Y32[:, [0]], k, "omp", tol=1e-4)
        o = run_oracle(A64, Y64[:, [0]], k, "omp", tol=1e-4)
        assert g["support"][0, 0] == o["support"][0, 0]
        if k == 1:
            compare(g, o)


def test_duplicate_atom_tie_and_dependent(cs_gpu, torch):
    rng = np.random.default_rng(22)
    A = workloads.gaussian_matrix(rng, 12, 30)
    A[:, 17] = A[:, 5]
    Y = np.stack([3.0 * A[:, 5] + 0.5 * A[:, 9], A[:, 5] * 2.0], axis=1)
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = run_gpu(cs_gpu, torch, A32, Y32, 2, "omp", tol=1e-3)
    assert g["support"][0, 0] == 5 and g["support"][1, 0] == 5
    assert g["status"][1] == 1 and g["n_iter"][1] == 1


def test_empty_batch_and_errors(cs_gpu, torch):
    A = torch.randn(16, 40, device="cuda")
    Y = torch.empty(16, 0, device="cuda")
    r = cs_gpu.omp_solve_batched(A, Y, 4)
    assert r.support.shape == (0, 4)
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.omp_solve_batched(A, torch.randn(16, 3, device="cuda"), 17)
    assert e.value.code == -1
    with pytest.raises(cs_gpu.CSError):
        cs_gpu.clomp_solve_batched(A, torch.randn(16, 3, device="cuda"), 4, beta1=1.5)


def test_batch_invariance_bitwise(cs_gpu, torch):
    """Eq. 3: columns sharing A are independent problems -- solving a batch
    equals solving each signal alone, bit for bit."""
    p = workloads.random_problem(64, 200, 40, 10, seed=23, snr_db=40.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    for algo in ("omp", "clomp"):
        full = run_gpu(cs_gpu, torch, A32, Y32, 10, algo)
        for b in (0, 7, 39):
            one = run_gpu(cs_gpu, torch, A32, Y32[:, [b]], 10, algo)
            assert np.array_equal(one["support"][0], full["support"][b])
            assert np.array_equal(one["coef"][0], full["coef"][b])


def test_host_entry_points_match_device(cs_gpu, torch):
    p = workloads.random_problem(48, 150, 64, 8, seed=24, snr_db=40.0)
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    for algo in ("omp", "clomp"):
        dev = run_gpu(cs_gpu, torch, A32, Y32, 8, algo)
        fn = cs_gpu.omp_solve_batched_host if algo == "omp" else cs_gpu.clomp_solve_batched_host
        host = fn(A32, Y32, 8)
        for q in ("support", "coef", "n_iter", "status"):
            assert np.array_equal(host[q], dev[q]), q


def test_clomp_reset_adam_option(cs_gpu, torch):
    p = workloads.random_problem(40, 120, 50, 6, seed=25, snr_db=40.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = run_gpu(cs_gpu, torch, A32, Y32, 6, "clomp", reset_adam=True, steps=30, lr=2e-2)
    o = run_oracle(A64, Y64, 6, "clomp", reset_adam=True, steps=30, lr=2e-2)
    compare(g, o)


@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_graph_replay_matches_eager(cs_gpu, torch, algo):
    """Repeated solves on one plan run eagerly, then as a captured CUDA graph;
    replays read the buffers' current contents and match eager runs bit for bit."""
    rng = np.random.default_rng(61)
    A = workloads.gaussian_matrix(rng, 64, 200)
    X1 = workloads.sparse_coefficients(rng, 200, 300, 10, values="pm")
    X2 = workloads.sparse_coefficients(rng, 200, 300, 10, values="pm")
    A32, Y1, _, _ = f32_problem(A, A @ X1)
    _, Y2, _, _ = f32_problem(A, A @ X2)
    At = _dev(torch, A32)
    Y = _dev(torch, Y1)
    plan = cs_gpu.Plan(64, 200, 300, 10)
    out = cs_gpu._outputs(300, 10, At.device)
    solve = (lambda: cs_gpu.omp_solve_batched(At, Y, 10, prec="bf16", plan=plan, out=out)) if algo == "omp" \
        else (lambda: cs_gpu.clomp_solve_batched(At, Y, 10, prec="bf16", plan=plan, out=out, **CL))
    got = []
    for Yh in (Y1, Y2, Y1, Y2):          # eager, capture + replay, replay, replay
        Y.copy_(torch.from_numpy(Yh))
        solve()
        torch.cuda.synchronize()
        got.append({q: v.clone() for q, v in vars(out).items()})
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert torch.equal(got[0][q], got[2][q]), q
        assert torch.equal(got[1][q], got[3][q]), q
    # the captured run equals an eager run on a fresh plan
    fresh = run_gpu(cs_gpu, torch, A32, Y2, 10, algo, prec="bf16", **({} if algo == "omp" else CL))
    assert np.array_equal(fresh["support"], got[1]["support"].cpu().numpy())
    assert np.array_equal(fresh["coef"], got[1]["coef"].cpu().numpy())


@pytest.mark.parametrize("algo,prec", [("omp", "fp32"), ("omp", "bf16"), ("clomp", "bf16"), ("clomp", "fp32")])
def test_same_bits_with_and_without_gram_table(cs_gpu, torch, algo, prec):
    """A plan sized for n <= 4096 keeps A^T A and reads Gram entries from
    it; a larger plan forms them from the columns.  Both give the same bits
    (the table is built in the selection's own dot-product arithmetic), and
    so does the process-wide default plan whatever sizes it grew to."""
    p = workloads.random_problem(96, 700, 300, 12, seed=64, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    kw = {} if algo == "omp" else dict(form="gram", **CL)
    small = run_gpu(cs_gpu, torch, A32, Y32, 12, algo, prec=prec, plan=cs_gpu.Plan(96, 700, 300, 12), **kw)
    big = run_gpu(cs_gpu, torch, A32, Y32, 12, algo, prec=prec, plan=cs_gpu.Plan(96, 5000, 300, 12), **kw)
    dflt = run_gpu(cs_gpu, torch, A32, Y32, 12, algo, prec=prec, **kw)
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(small[q], big[q]), q
        assert np.array_equal(small[q], dflt[q]), q


def test_fused_update_matches_separate_kernels(cs_gpu, torch):
    """The fused CLOMP update (selection + fit + residual in one kernel) runs
    the same per-signal arithmetic as the three separate kernels."""
    p = workloads.random_problem(77, 301, 333, 20, seed=71, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = _dev(torch, A32)
    Y = _dev(torch, Y32)
    res = []
    for fuse in (1, 0):
        plan = cs_gpu.Plan(77, 301, 333, 20)
        plan.set_option(cs_gpu.OPT_FUSE_UPDATE, fuse)
        r = cs_gpu.clomp_solve_batched(A, Y, 20, prec="bf16", plan=plan, **CL)
        plan.profile(reset=False)
        torch.cuda.synchronize()
        res.append(to_numpy(r))
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(res[0][q], res[1][q]), q
