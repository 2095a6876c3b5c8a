"""Batched IHT (the paper's comparison method) on the float32 correlation
kernel, against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from parity import COEF_RTOL, AMBIGUOUS_MARGIN, f32_problem, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def run(cs, torch, A32, Y32, k, step, **kw):
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = kw.pop("plan", None) or cs.Plan(A32.shape[0], A32.shape[1], Y32.shape[1], k)
    r = cs.iht_solve_batched(A, Y, k, step, plan=plan, **kw)
    torch.cuda.synchronize()
    return to_numpy(r)


def compare_iht(g, o):
    """Kept sets identical (ascending), coefficients within COEF_RTOL,
    iterations and status equal -- unless the oracle's own k-th/(k+1)-th gap
    fell below AMBIGUOUS_MARGIN at some iteration (float32 cannot resolve
    the kept set there), which is counted and must stay rare."""
    ambiguous, worst = 0, 0.0
    for b in range(o["support"].shape[0]):
        if not np.array_equal(g["support"][b], o["support"][b]):
            assert o["margin"][b] < AMBIGUOUS_MARGIN, (b, o["margin"][b], g["support"][b], o["support"][b])
            ambiguous += 1
            continue
        assert g["n_iter"][b] == o["n_iter"][b] and g["status"][b] == o["status"][b], b
        nrm = np.linalg.norm(o["coef"][b])
        err = np.linalg.norm(g["coef"][b] - o["coef"][b]) / (nrm if nrm > 0 else 1.0)
        worst = max(worst, err)
        assert err <= COEF_RTOL, (b, err)
    assert ambiguous <= max(1, o["support"].shape[0] // 100)
    return dict(signals=o["support"].shape[0], ambiguous=ambiguous, max_coef_rel_err=worst)


@pytest.mark.parametrize("m,n,B,k,it,snr", [(256, 1024, 512, 32, 200, 40.0),   # the batched workload's shape
                                            (77, 301, 133, 12, 60, 30.0)])     # ragged
def test_iht_matches_oracle(cs_gpu, torch, m, n, B, k, it, snr):
    p = workloads.random_problem(m, n, B, k, seed=m + B, snr_db=snr, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    step = float(np.float32(1.0 / np.linalg.norm(A64, 2) ** 2))
    g = run(cs_gpu, torch, A32, Y32, k, step, max_iter=it)
    o = oracle.iht(A64, Y64, k, step, max_iter=it)
    print(compare_iht(g, o))


def test_iht_stop_rules_and_graph_replay(cs_gpu, torch):
    rng = np.random.default_rng(97)
    A = workloads.gaussian_matrix(rng, 48, 160)
    X = workloads.sparse_coefficients(rng, 160, 5, 4)
    Y = A @ X
    Y[7, 1] = np.nan
    Y[:, 2] = 0.0
    A32, Y32, A64, Y64 = f32_problem(A, Y)
    step = float(np.float32(1.0 / np.linalg.norm(A64, 2) ** 2))
    plan = cs_gpu.Plan(48, 160, 5, 4)
    runs = [run(cs_gpu, torch, A32, Y32, 4, step, max_iter=400, tol=1e-4, plan=plan) for _ in range(3)]
    for r in runs[1:]:           # eager, captured, replayed: the same bits
        for q in r:
            assert np.array_equal(r[q], runs[0][q], equal_nan=True), q
    g = runs[0]
    o = oracle.iht(A64, Y64, 4, step, max_iter=400, tol=1e-4)
    assert g["status"][1] == 4 and g["n_iter"][1] == 0
    assert g["status"][2] == 1 and g["n_iter"][2] == 0 and np.all(g["support"][2] == -1)
    for b in (0, 3, 4):
        assert g["support"][b].tolist() == o["support"][b].tolist()
        assert g["status"][b] == o["status"][b]
        assert abs(int(g["n_iter"][b]) - int(o["n_iter"][b])) <= 1     # tol crossed within one step


def test_iht_limits(cs_gpu, torch):
    A = torch.randn(64, 5000, device="cuda")
    Y = torch.randn(64, 2, device="cuda")
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.iht_solve_batched(A, Y, 8, 0.01)
    assert e.value.code == -5
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.iht_solve_batched(A[:, :100], Y, 8, -1.0)
    assert e.value.code == -1
