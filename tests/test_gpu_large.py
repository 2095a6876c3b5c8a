"""The large-instance OMP path (supports beyond the on-chip 64 atoms, more
than 1024 rows, the bf16 correlation beyond the tensor-core kernel's sizes)
against the FP64 oracle, through the C ABI (via the ctypes binding)."""
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


def run(cs, torch, A32, Y32, k, prec, plan=None, **kw):
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    m, n = A32.shape
    plan = plan or cs.Plan(m, n, Y32.shape[1], k)
    r = cs.omp_solve_batched(A, Y, k, prec=prec, plan=plan, **kw)
    torch.cuda.synchronize()
    g = to_numpy(r)
    g["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    return g


def large_signal(n, m, k, seed):
    """A noiseless k-sparse signal with N(0,1) values in a Gaussian dictionary
    with unit columns (the large 1-D workload's recipe at a smaller size)."""
    rng = np.random.default_rng(seed)
    A = workloads.gaussian_matrix(rng, m, n)
    X = workloads.sparse_coefficients(rng, n, 1, k, values="gauss")
    return A, A @ X, X


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_large_signal_full_length(cs_gpu, torch, prec):
    """n = 16384, m = 4915, k = 500 (the large 1-D workload scaled down by 4
    in n and m), all 500 iterations against the incremental-QR oracle, and
    exact recovery of the noiseless signal."""
    A, Y, X = large_signal(16384, 4915, 500, seed=401)
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = run(cs_gpu, torch, A32, Y32, 500, prec)
    o = oracle.omp(A64, Y64, 500)
    s = compare(g, o)
    print(prec, s)
    assert g["status"][0] == 0 and g["n_iter"][0] == 500
    truth = np.nonzero(X[:, 0])[0]
    assert sorted(g["support"][0].tolist()) == sorted(truth.tolist())
    xr = np.zeros(A.shape[1])
    xr[g["support"][0]] = g["coef"][0]
    assert np.linalg.norm(xr - X[:, 0]) <= 1e-5 * np.linalg.norm(X[:, 0])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("m,n,B,k,snr", [(300, 1000, 5, 100, 30.0),      # k beyond the on-chip 64
                                         (1500, 3001, 3, 20, 40.0),      # more rows than a warp holds
                                         (333, 1203, 7, 40, 30.0),       # bf16 beyond the tensor-core sizes
                                         (150, 301, 9, 65, 20.0)])       # ragged, k near m / 2
def test_large_path_matches_oracle(cs_gpu, torch, prec, m, n, B, k, snr):
    p = workloads.random_problem(m, n, B, k, seed=m + n + k, snr_db=snr, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = run(cs_gpu, torch, A32, Y32, k, prec)
    s = compare(g, oracle.omp(A64, Y64, k))
    print(prec, m, n, B, k, s)


def test_large_path_stop_rules_and_edges(cs_gpu, torch):
    """Non-finite input (status 4), a zero signal under tol (1), max_iter (2),
    a duplicated atom (tie to the lower index)."""
    rng = np.random.default_rng(402)
    m, n, k = 120, 400, 80
    A = workloads.gaussian_matrix(rng, m, n)
    A[:, 250] = A[:, 17]
    Y = rng.standard_normal((m, 4))
    Y[5, 1] = np.nan
    Y[:, 2] = 0.0
    Y[:, 3] = 3.0 * A[:, 17] + 0.25 * A[:, 90]
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    g = run(cs_gpu, torch, A32, Y32, k, "fp32", max_iter=60, tol=1e-3)
    o = oracle.omp(A64, Y64, k, max_iter=60, tol=1e-3)
    assert g["status"].tolist()[:3] == [2, 4, 1]
    assert g["n_iter"].tolist()[:3] == [60, 0, 0]
    assert g["support"][3, 0] == 17
    compare({q: v[[0]] for q, v in g.items() if q != "launches"},
            {q: v[[0]] for q, v in o.items()})
    # y on atom 17 alone: the tie with its copy goes to 17, then the exact
    # fit stops on tol after one atom
    y = np.float32(A32[:, 17] * 2.0)
    g = run(cs_gpu, torch, A32, y.reshape(-1, 1), 70, "fp32", tol=1e-3)
    assert g["support"][0, 0] == 17 and g["status"][0] == 1 and g["n_iter"][0] == 1


def test_large_path_deterministic_and_routed(cs_gpu, torch):
    """Two solves give the same bits; the large path runs its own launch
    groups (one correlation, selection, least-squares and residual group per
    iteration, none of the on-chip kernels)."""
    p = workloads.random_problem(400, 2000, 4, 90, seed=403, snr_db=30.0)
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    a = run(cs_gpu, torch, A32, Y32, 90, "bf16")
    b = run(cs_gpu, torch, A32, Y32, 90, "bf16")
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(a[q], b[q]), q
    ln = a["launches"]
    assert ln["correlation"] == ln["select"] == ln["fit"] == ln["residual"] == 90
    assert ln["persist"] == 0 and ln["update"] == 0 and ln["setup"] == 1


def _oracle_clomp(A64, Y64, k, **kw):
    f = lambda v: float(np.float32(v))
    return oracle.clomp(A64, Y64, k, steps=50, lr=f(1e-2), beta1=f(0.9), beta2=f(0.999), eps=f(1e-8), **kw)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("m,n,B,k,snr", [(2048, 8192, 1, 150, None),     # one long noiseless signal
                                         (300, 1000, 4, 100, 30.0),      # k beyond the on-chip 64
                                         (1500, 3001, 3, 20, 40.0)])     # more rows than a warp holds
def test_large_path_clomp_matches_oracle(cs_gpu, torch, prec, m, n, B, k, snr):
    """CLOMP in Gram form on the large-instance path (G and b grown per
    iteration, 50 Adam steps per iteration, one Adam state for the solve)."""
    p = workloads.random_problem(m, n, B, k, seed=m + 3 * k, snr_db=snr, values="gauss" if snr is None else "pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = cs_gpu.Plan(m, n, B, k)
    r = cs_gpu.clomp_solve_batched(A, Y, k, prec=prec, form="gram", plan=plan, steps=50, lr=1e-2)
    torch.cuda.synchronize()
    g = to_numpy(r)
    ln = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    assert ln["persist"] == 0 and ln["update"] == 0 and ln["correlation"] == k
    assert plan.counters(reset=True)[1] == 0
    print(prec, m, n, B, k, compare(g, _oracle_clomp(A64, Y64, k)))


def test_large_path_clomp_reset_adam(cs_gpu, torch):
    """reset_adam_each_iter on the large-instance path: the moments and the
    step counter restart at every iteration.  Supports identical; the
    coefficients within 1e-3, not 1e-5: every restart's first steps move each
    coordinate by about lr sign(g), and for coordinates already at their
    optimum g is at float32 rounding level, so its sign is noise.  The same
    steps in numpy float32 differ from the FP64 oracle by 2.6e-4 to 3.4e-4
    here (in float64 by 1e-13); without the reset the moments keep these
    steps small (2e-7)."""
    p = workloads.random_problem(1100, 2000, 3, 40, seed=77, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    r = cs_gpu.clomp_solve_batched(torch.from_numpy(np.asfortranarray(A32)).cuda(),
                                   torch.from_numpy(np.asfortranarray(Y32)).cuda(), 40, form="gram",
                                   plan=cs_gpu.Plan(1100, 2000, 3, 40), steps=50, lr=1e-2, reset_adam=True)
    torch.cuda.synchronize()
    print(compare(to_numpy(r), _oracle_clomp(A64, Y64, 40, reset_adam=True), coef_rtol=1e-3))


def test_large_path_clomp_many_signals(cs_gpu, torch):
    """More signals than the fit's cooperative launch can hold resident
    (1300 > 152 SMs x 8 CTAs): the fit runs one launch per Adam step; the
    results still match the oracle."""
    m, n, B, k = 1100, 1200, 1300, 3
    p = workloads.random_problem(m, n, B, k, seed=78, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    plan = cs_gpu.Plan(m, n, B, k)
    r = cs_gpu.clomp_solve_batched(torch.from_numpy(np.asfortranarray(A32)).cuda(),
                                   torch.from_numpy(np.asfortranarray(Y32)).cuda(), k, form="gram",
                                   plan=plan, steps=50, lr=1e-2)
    torch.cuda.synchronize()
    assert plan.counters(reset=True)[1] == 0
    print(compare(to_numpy(r), _oracle_clomp(A64, Y64, k)))


def test_large_path_clomp_refusals(cs_gpu, torch):
    """Beyond the on-chip sizes CLOMP runs the Gram form with one atom per
    iteration and no prior; the literal gather form is refused there."""
    A = torch.randn(300, 1000, device="cuda")
    Y = torch.randn(300, 2, device="cuda")
    plan = cs_gpu.Plan(300, 1000, 2, 100)
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 100, form="gather", plan=plan)
    assert e.value.code == -5
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.clomp_solve_batched(A, Y, 100, form="gram", plan=plan, th=0.7)
    assert e.value.code == -5


def _large_solve(cs, torch, A32, Y32, k, algo, prec="bf16"):
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    m, n = A32.shape
    plan = cs.Plan(m, n, Y32.shape[1], k)
    if algo == "omp":
        r = cs.omp_solve_batched(A, Y, k, prec=prec, plan=plan)
    else:
        r = cs.clomp_solve_batched(A, Y, k, prec=prec, form="gram", plan=plan, steps=50, lr=1e-2)
    torch.cuda.synchronize()
    g = to_numpy(r)
    assert plan.counters(reset=True)[1] == 0
    return g


@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_large_path_gemm_correlation_same_bits(cs_gpu, torch, algo):
    """Eight or more signals sharing A (bf16) correlate as one tensor-core
    GEMM over bf16 residuals; fewer stream A once per pass.  Both lists are
    certified and re-scored in float32, so the float32 argmax -- and every
    output -- is the same: 40 signals solved as one group and as ten groups
    of four give the same bits (n and m not multiples of the tile sizes)."""
    m, n, B, k = 1100, 3001, 40, 60
    p = workloads.random_problem(m, n, B, k, seed=501, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    one = _large_solve(cs_gpu, torch, A32, Y32, k, algo)
    parts = [_large_solve(cs_gpu, torch, A32, np.asfortranarray(Y32[:, i:i + 4]), k, algo) for i in range(0, B, 4)]
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(one[q], np.concatenate([g[q] for g in parts], axis=0)), q
    o = oracle.omp(A64, Y64, k) if algo == "omp" else _oracle_clomp(A64, Y64, k)
    print(algo, compare(one, o))


def test_large_path_gemm_correlation_two_passes(cs_gpu, torch):
    """300 signals: the GEMM runs two passes (256 and 44 signals)."""
    m, n, B, k = 1030, 1500, 300, 8
    p = workloads.random_problem(m, n, B, k, seed=502, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = _large_solve(cs_gpu, torch, A32, Y32, k, "omp")
    print(compare(g, oracle.omp(A64, Y64, k)))


def test_large_path_gemm_correlation_edges(cs_gpu, torch):
    """The GEMM correlation's group (10 signals, bf16) with a NaN signal
    (status 4: its residual column is NaN but no other signal's is touched),
    a zero signal under tol (1), max_iter (2) and a duplicated atom (the tie
    to the lower index): the same bits as the signals solved in groups of
    fewer than eight (streaming), and the oracle's results."""
    rng = np.random.default_rng(503)
    m, n, k = 1100, 900, 40
    A = workloads.gaussian_matrix(rng, m, n)
    A[:, 610] = A[:, 23]
    X = workloads.sparse_coefficients(rng, n, 10, 12, values="pm")
    Y = A @ X + 0.01 * rng.standard_normal((m, 10))
    Y[5, 1] = np.nan
    Y[:, 2] = 0.0
    Y[:, 3] = 3.0 * A[:, 23] + 0.25 * A[:, 90]
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    Am = torch.from_numpy(np.asfortranarray(A32)).cuda()

    def solve(cols):
        Yc = torch.from_numpy(np.asfortranarray(Y32[:, cols])).cuda()
        r = cs_gpu.omp_solve_batched(Am, Yc, k, prec="bf16", plan=cs_gpu.Plan(m, n, len(cols), k), tol=1e-3,
                                     max_iter=30)
        torch.cuda.synchronize()
        return to_numpy(r)

    one = solve(list(range(10)))
    a, b = solve(list(range(5))), solve(list(range(5, 10)))
    for q in ("support", "coef", "n_iter", "status"):
        assert np.array_equal(one[q], np.concatenate([a[q], b[q]], axis=0)), q
    assert np.array_equal(one["res_norm"], np.concatenate([a["res_norm"], b["res_norm"]]), equal_nan=True)
    assert one["status"][1] == 4 and one["status"][2] == 1 and one["support"][3, 0] == 23
    assert one["status"][0] == 2 and one["n_iter"][0] == 30
    ok = [0, 3, 4, 5, 6, 7, 8, 9]
    o = oracle.omp(A64, Y64[:, ok], k, tol=1e-3, max_iter=30)
    compare({q: v[ok] for q, v in one.items()}, o)
