"""Pins of the FP64 oracle against facts other than its own code.

Each test would fail on a plausible mistake in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong tie-break or stop rule):
  * brute-force support search on tiny noiseless instances, with the Exact
    Recovery Condition deciding where OMP must succeed;
  * orthogonality of the least-squares residual to the selected atoms;
  * monotone residual norm;
  * orthonormal A: closed form of every OMP step;
  * Householder-QR least squares vs numpy.linalg.lstsq (library);
  * exact recovery on the single-signal workload;
  * hand-derived worked examples stored under tests/golden/;
  * CL gradient vs central finite differences of the quadratic loss;
  * the CL Adam loop vs torch.optim.Adam in float64 (library);
  * orthonormal A decouples the CL fit coordinate by coordinate;
  * the CL fit approaches the least-squares coefficients for long, small-step runs;
  * threshold (Th) selection: closed-form sets, order and margin on an
    orthonormal dictionary over several iterations, the k cap, and Th -> 1
    reducing to the argmax rule.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_A(rng, m, n):
    return workloads.gaussian_matrix(rng, m, n)


# ---------------------------------------------------------------- OMP pins

def test_lstsq_matches_numpy():
    rng = np.random.default_rng(1)
    for (m, t) in [(8, 1), (16, 5), (64, 20), (256, 32), (33, 33)]:
        As = rng.standard_normal((m, t))
        y = rng.standard_normal(m)
        z, st = oracle.lstsq(As, y)
        assert st == 0
        z_ref = np.linalg.lstsq(As, y, rcond=None)[0]
        assert np.allclose(z, z_ref, rtol=1e-12, atol=1e-12 * np.abs(z_ref).max())


def test_lstsq_flags_dependent_column():
    rng = np.random.default_rng(2)
    As = rng.standard_normal((10, 3))
    As = np.column_stack([As, As[:, 0] * 2.0 - As[:, 2]])
    _, st = oracle.lstsq(As, rng.standard_normal(10))
    assert st == 3


def _erc_holds(A, S):
    """Tropp's Exact Recovery Condition max_{j not in S} ||pinv(A_S) a_j||_1 < 1."""
    P = np.linalg.pinv(A[:, S])
    others = [j for j in range(A.shape[1]) if j not in S]
    return max(np.abs(P @ A[:, j]).sum() for j in others) < 1.0


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_bruteforce_tiny_noiseless(method):
    """n <= 20, k <= 3: the minimum-residual support over all C(n,k) supports
    is the true one, and OMP recovers it wherever the ERC holds."""
    rng = np.random.default_rng(3)
    n_erc = 0
    for trial in range(60):
        m, n, k = int(rng.integers(6, 13)), int(rng.integers(10, 21)), int(rng.integers(1, 4))
        A = _rand_A(rng, m, n)
        S_true = sorted(rng.choice(n, size=k, replace=False).tolist())
        x = np.zeros(n)
        x[S_true] = rng.standard_normal(k) + np.sign(rng.standard_normal(k))
        y = A @ x
        best, best_res = None, np.inf
        for S in itertools.combinations(range(n), k):
            z = np.linalg.lstsq(A[:, S], y, rcond=None)[0]
            res = np.linalg.norm(y - A[:, S] @ z)
            if res < best_res - 1e-12:
                best, best_res = list(S), res
        assert best == S_true
        o = oracle.omp(A, y, k, tol=0.0, method=method)
        if _erc_holds(A, S_true):
            n_erc += 1
            assert sorted(o["support"][0].tolist()) == S_true
            xr = np.zeros(n)
            xr[o["support"][0]] = o["coef"][0]
            assert np.allclose(xr, x, atol=1e-10)
    assert n_erc >= 10


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_residual_orthogonal_and_monotone(method):
    rng = np.random.default_rng(4)
    A = _rand_A(rng, 48, 160)
    X = workloads.sparse_coefficients(rng, 160, 6, 10, values="gauss")
    Y = workloads.add_noise(rng, A @ X, 30.0)
    for kk in range(1, 11):
        o = oracle.omp(A, Y, kk, method=method)
        for b in range(Y.shape[1]):
            S = o["support"][b]
            r = Y[:, b] - A[:, S] @ o["coef"][b]
            bound = 1e-10 * np.linalg.norm(A[:, S], 2) * np.linalg.norm(Y[:, b])
            assert np.abs(A[:, S].T @ r).max() <= bound
            assert abs(np.linalg.norm(r) - o["res_norm"][b]) <= 1e-12 * np.linalg.norm(Y[:, b])
    h = o["res_hist"]
    assert np.all(np.diff(h, axis=1) <= 1e-12)


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_orthonormal_closed_form(method):
    """A orthonormal (m = n): supports come in descending |A^T y| order, the
    coefficients are (A^T y)_S and ||r||^2 = ||y||^2 - sum of selected c^2."""
    rng = np.random.default_rng(5)
    n = 24
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Y = rng.standard_normal((n, 3))
    k = 7
    o = oracle.omp(Q, Y, k, method=method)
    for b in range(3):
        c = Q.T @ Y[:, b]
        order = np.argsort(-np.abs(c), kind="stable")[:k]
        assert o["support"][b].tolist() == order.tolist()
        assert np.allclose(o["coef"][b], c[order], atol=1e-12)
        rr = np.sum(Y[:, b] ** 2) - np.sum(c[order] ** 2)
        assert abs(o["res_norm"][b] ** 2 - rr) < 1e-10
        for t in range(k):   # the logged top-1 is |c| of the pick itself
            assert abs(o["top1"][b, t] - abs(c[order[t]])) < 1e-12


def test_single_signal_exact_recovery():
    p = workloads.config_single_fp64()
    o = oracle.omp(p.A, p.Y, p.k, tol=p.tol)
    xr = np.zeros(p.n)
    xr[o["support"][0]] = o["coef"][0]
    assert sorted(o["support"][0].tolist()) == sorted(np.nonzero(p.X_true[:, 0])[0].tolist())
    assert np.abs(xr - p.X_true[:, 0]).max() < 1e-10
    assert o["status"][0] == 1 and o["n_iter"][0] == 8


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_tie_lowest_index_and_dependent_atom(method):
    rng = np.random.default_rng(6)
    A = _rand_A(rng, 12, 30)
    A[:, 17] = A[:, 5]                     # duplicated atom
    y = 3.0 * A[:, 5] + 0.5 * A[:, 9]
    o = oracle.omp(A, y, 2, method=method)
    assert o["support"][0, 0] == 5         # exact tie 5/17 -> lowest index
    assert o["top2"][0, 0] == o["top1"][0, 0]
    # more atoms than measurements can carry: the 13th column is dependent
    Y = rng.standard_normal((12, 1))
    o = oracle.omp(A, Y, 12, tol=0.0, method=method)
    assert o["status"][0] in (0, 3)
    B2 = _rand_A(rng, 4, 8)
    B2[:, 1] = B2[:, 0]
    B2[:, 2] = B2[:, 0]
    y2 = B2[:, 0] * 2.0
    o = oracle.omp(B2, y2, 3, tol=0.0, method=method)
    # after picking atom 0 the residual is 0; the next pick is dependent
    assert o["status"][0] == 3 and o["n_iter"][0] == 1 and o["support"][0, 0] == 0


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_nonfinite_and_stop_rules(method):
    rng = np.random.default_rng(7)
    A = _rand_A(rng, 16, 40)
    Y = rng.standard_normal((16, 4))
    Y[3, 1] = np.nan
    Y[:, 2] = 0.0
    o = oracle.omp(A, Y, 5, tol=1e-9, max_iter=3, method=method)
    assert o["status"].tolist() == [2, 4, 1, 2]
    assert o["n_iter"].tolist() == [3, 0, 0, 3]
    assert np.all(o["support"][1] == -1)
    o = oracle.omp(A, Y[:, [0]], 5, tol=0.0, max_iter=5, method=method)
    assert o["status"][0] == 0 and o["n_iter"][0] == 5


@pytest.mark.parametrize("method", ["householder", "iqr"])
def test_batch_invariance_and_leading_dims(method):
    rng = np.random.default_rng(8)
    A = _rand_A(rng, 20, 50)
    Y = rng.standard_normal((20, 5))
    o_all = oracle.omp(A, Y, 6, method=method)
    for b in range(5):
        o1 = oracle.omp(A, Y[:, b], 6, method=method)
        assert np.array_equal(o1["support"][0], o_all["support"][b])
        assert np.array_equal(o1["coef"][0], o_all["coef"][b])


def test_iqr_matches_householder_on_larger_supports():
    """The incremental QR (modified Gram-Schmidt, twice) and the Householder
    QR recomputed every iteration are different algorithms for the same
    least-squares fits: same supports, coefficients to 1e-11, on noisy
    signals with supports of 100 atoms."""
    rng = np.random.default_rng(31)
    A = _rand_A(rng, 300, 900)
    X = workloads.sparse_coefficients(rng, 900, 3, 100, values="gauss")
    Y = workloads.add_noise(rng, A @ X, 30.0)
    a = oracle.omp(A, Y, 100, method="householder")
    b = oracle.omp(A, Y, 100, method="iqr")
    assert np.array_equal(a["support"], b["support"])
    for q in range(3):
        assert np.linalg.norm(a["coef"][q] - b["coef"][q]) <= 1e-11 * np.linalg.norm(a["coef"][q])
    assert np.allclose(a["res_norm"], b["res_norm"], rtol=1e-11)


def test_iqr_large_noiseless_exact_recovery_single_signal():
    """A noiseless k-sparse signal with m well above 2 k log(n/k): the
    incremental-QR oracle (one signal, atoms split over threads) recovers the
    support and the coefficients to 1e-9, its residual is orthogonal to the
    selected atoms, and the result equals the same signal solved inside a
    batch (signals split over threads)."""
    rng = np.random.default_rng(32)
    m, n, k = 600, 2400, 120
    A = _rand_A(rng, m, n)
    X = workloads.sparse_coefficients(rng, n, 2, k, values="gauss")
    Y = A @ X
    o1 = oracle.omp(A, Y[:, 0], k, method="iqr")
    assert sorted(o1["support"][0].tolist()) == sorted(np.nonzero(X[:, 0])[0].tolist())
    xr = np.zeros(n)
    xr[o1["support"][0]] = o1["coef"][0]
    assert np.abs(xr - X[:, 0]).max() <= 1e-9 * np.abs(X[:, 0]).max()
    S = o1["support"][0]
    r = Y[:, 0] - A[:, S] @ o1["coef"][0]
    assert np.abs(A[:, S].T @ r).max() <= 1e-10 * np.linalg.norm(A[:, S], 2) * np.linalg.norm(Y[:, 0])
    o2 = oracle.omp(A, Y, k, method="iqr")
    assert np.array_equal(o2["support"][0], o1["support"][0])
    assert np.array_equal(o2["coef"][0], o1["coef"][0])


def test_golden_worked_examples():
    """Hand-derived OMP runs (see the derivations inside each fixture)."""
    for fn in sorted(os.listdir(GOLDEN)):
        if not fn.startswith("omp_") or not fn.endswith(".json"):
            continue
        g = json.load(open(os.path.join(GOLDEN, fn)))
        A = np.array(eval_expr(g["A"]), dtype=np.float64)
        y = np.array(eval_expr(g["y"]), dtype=np.float64)
        o = oracle.omp(A, y, g["k"], tol=g["tol"])
        assert o["support"][0].tolist() == g["support"], fn
        assert np.allclose(o["coef"][0], eval_expr(g["coef"]), atol=1e-14), fn
        assert o["status"][0] == g["status"], fn


def eval_expr(v):
    """Fixture numbers may be written as closed forms such as "sqrt(3)"."""
    if isinstance(v, list):
        return [eval_expr(u) for u in v]
    if isinstance(v, str):
        return float(eval(v, {"__builtins__": {}}, {"sqrt": math.sqrt}))
    return float(v)


# ---------------------------------------------------------------- CLOMP pins

def test_clfit_gradient_matches_central_differences():
    """L is quadratic in s_S, so a central difference has no truncation error."""
    rng = np.random.default_rng(9)
    A = _rand_A(rng, 40, 90)
    S = rng.choice(90, size=7, replace=False).astype(np.int32)
    y = rng.standard_normal(40)
    s = rng.standard_normal(7)
    L0, g, r = oracle.clfit_loss_grad(A, S, s, y)
    assert abs(L0 - 0.5 * np.sum((y - A[:, S] @ s) ** 2)) < 1e-12
    h = 1e-3
    for q in range(7):
        e = np.zeros(7)
        e[q] = h
        Lp = oracle.clfit_loss_grad(A, S, s + e, y)[0]
        Lm = oracle.clfit_loss_grad(A, S, s - e, y)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-9 * max(1.0, abs(g[q]))


def test_clfit_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    A = _rand_A(rng, 32, 64)
    S = np.array([3, 17, 40, 41, 60], dtype=np.int32)
    y = rng.standard_normal(32)
    s0 = np.zeros(5)
    s_o, mo, ve, tau = oracle.clfit_adam(A, S, y, s0, np.zeros(5), np.zeros(5), 0, 300,
                                         lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    assert tau == 300
    At = torch.tensor(A[:, S], dtype=torch.float64)
    yt = torch.tensor(y, dtype=torch.float64)
    p = torch.zeros(5, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    for _ in range(300):
        opt.zero_grad()
        loss = 0.5 * torch.sum((yt - At @ p) ** 2)
        loss.backward()
        opt.step()
    assert np.allclose(s_o, p.detach().numpy(), rtol=0, atol=1e-13)
    st = opt.state[p]
    assert np.allclose(mo, st["exp_avg"].numpy(), atol=1e-13)
    assert np.allclose(ve, st["exp_avg_sq"].numpy(), atol=1e-13)


def test_clomp_first_iteration_is_adam_on_growing_mask():
    """CLOMP iteration structure: with steps T the state after t iterations is
    the state of one Adam run (torch) on the masked loss whose mask grows by
    the oracle's picks, T steps per pick (one optimizer state for the solve)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    A = _rand_A(rng, 24, 60)
    X = workloads.sparse_coefficients(rng, 60, 1, 4, values="pm")
    y = (A @ X)[:, 0]
    T, k = 20, 4
    o = oracle.clomp(A, y, k, steps=T, lr=5e-2)
    S = o["support"][0]
    p = torch.zeros(60, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=5e-2, foreach=False)
    At = torch.tensor(A, dtype=torch.float64)
    yt = torch.tensor(y, dtype=torch.float64)
    mask = torch.zeros(60, dtype=torch.float64)
    r = yt.clone()
    for t in range(k):
        c = (At.T @ r).abs().numpy()
        c[mask.numpy() > 0] = -1
        assert int(np.argmax(c)) == S[t]
        mask[S[t]] = 1.0
        for _ in range(T):
            opt.zero_grad()
            loss = 0.5 * torch.sum((yt - At @ (p * mask)) ** 2)
            loss.backward()
            opt.step()
        with torch.no_grad():
            r = yt - At @ (p * mask)
    assert np.allclose(p.detach().numpy()[S], o["coef"][0], atol=1e-12)
    assert abs(float(torch.linalg.norm(r)) - o["res_norm"][0]) < 1e-12


def test_clomp_reset_adam_is_a_fresh_optimizer_per_pick():
    """The restart option: every iteration starts a new Adam (moments zero,
    step counter back at 1) on the grown mask, while the coefficients carry
    over -- a fresh torch optimizer per pick on the same parameter.  Its
    result differs from the single-optimizer run, so the option matters."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(14)
    A = _rand_A(rng, 24, 60)
    X = workloads.sparse_coefficients(rng, 60, 1, 4, values="pm")
    y = (A @ X)[:, 0]
    T, k = 20, 4
    o = oracle.clomp(A, y, k, steps=T, lr=5e-2, reset_adam=True)
    S = o["support"][0]
    p = torch.zeros(60, dtype=torch.float64, requires_grad=True)
    At = torch.tensor(A, dtype=torch.float64)
    yt = torch.tensor(y, dtype=torch.float64)
    mask = torch.zeros(60, dtype=torch.float64)
    r = yt.clone()
    for t in range(k):
        c = (At.T @ r).abs().numpy()
        c[mask.numpy() > 0] = -1
        assert int(np.argmax(c)) == S[t]
        mask[S[t]] = 1.0
        opt = torch.optim.Adam([p], lr=5e-2, foreach=False)
        for _ in range(T):
            opt.zero_grad()
            loss = 0.5 * torch.sum((yt - At @ (p * mask)) ** 2)
            loss.backward()
            opt.step()
        with torch.no_grad():
            r = yt - At @ (p * mask)
    assert np.allclose(p.detach().numpy()[S], o["coef"][0], atol=1e-12)
    assert abs(float(torch.linalg.norm(r)) - o["res_norm"][0]) < 1e-12
    one = oracle.clomp(A, y, k, steps=T, lr=5e-2, reset_adam=False)
    assert np.max(np.abs(one["coef"][0] - o["coef"][0])) > 1e-6


def test_clomp_orthonormal_decouples():
    """With orthonormal A the CL gradient of coordinate q is s_q - c_q
    (c = A^T y): every coordinate runs its own scalar Adam on 1/2(s - c)^2."""
    rng = np.random.default_rng(12)
    n = 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    y = rng.standard_normal(n)
    c = Q.T @ y
    S = np.argsort(-np.abs(c))[:3].astype(np.int32)
    s, mo, ve, tau = oracle.clfit_adam(Q, S, y, np.zeros(3), np.zeros(3), np.zeros(3), 0, 40,
                                       lr=0.05)
    for q in range(3):
        s1, _, _, _ = oracle.clfit_adam(Q, S[[q]], y, [0.0], [0.0], [0.0], 0, 40, lr=0.05)
        assert abs(s1[0] - s[q]) < 1e-13
    _, g, _ = oracle.clfit_loss_grad(Q, S, s, y)
    assert np.allclose(g, s - c[S], atol=1e-13)


def test_clomp_long_small_steps_approach_least_squares():
    p = workloads.config_single_fp64()
    om = oracle.omp(p.A, p.Y, p.k, tol=0.0)
    cl = oracle.clomp(p.A, p.Y, p.k, tol=0.0, steps=20000, lr=1e-4, reset_adam=False)
    assert cl["support"][0].tolist() == om["support"][0].tolist()
    assert np.abs(cl["coef"][0] - om["coef"][0]).max() < 1e-3


def test_clomp_excludes_selected_and_stops():
    rng = np.random.default_rng(13)
    A = _rand_A(rng, 30, 80)
    Y = rng.standard_normal((30, 3))
    Y[0, 2] = np.inf
    o = oracle.clomp(A, Y, 10, steps=5)
    for b in range(2):
        assert len(set(o["support"][b].tolist())) == 10
        assert o["status"][b] == 0
    assert o["status"][2] == 4


def test_clomp_single_signal_parallel_correlation_matches_batch():
    """A single signal takes the correlation split over threads; its results
    equal the same signal solved inside a batch (serial correlation), bit for
    bit, including an exact tie (a duplicated column)."""
    rng = np.random.default_rng(17)
    A = _rand_A(rng, 40, 300)
    A[:, 201] = A[:, 7]
    Y = A[:, [7, 50, 120]] @ np.array([1.0, -0.5, 0.25])[:, None] + 0.01 * rng.standard_normal((40, 1))
    Y2 = np.concatenate([Y, rng.standard_normal((40, 1))], axis=1)
    one = oracle.clomp(A, Y, 12, steps=7, nthreads=4)
    two = oracle.clomp(A, Y2, 12, steps=7, nthreads=4)
    assert one["support"][0].tolist() == two["support"][0].tolist()
    assert 201 not in one["support"][0].tolist()[:1]
    for q in ("coef", "top1", "top2"):
        assert np.array_equal(one[q][0], two[q][0])


# ------------------------------------------------ threshold selection pins

def _threshold_sets(x, th, k):
    """Closed form of the threshold rule on an orthonormal dictionary:
    c_j = x_j for every unselected atom at every iteration, so each iteration
    takes the unselected atoms with |x_j| >= th * max, largest first."""
    chosen, sets = [], []
    ax = np.abs(x)
    while len(chosen) < k:
        rest = [j for j in range(len(x)) if j not in chosen]
        M = max(ax[j] for j in rest)
        it = sorted([j for j in rest if ax[j] >= th * M], key=lambda j: (-ax[j], j))
        it = it[: k - len(chosen)]
        sets.append(it)
        chosen += it
    return sets


def test_clomp_threshold_orthonormal_closed_form():
    """Orthonormal A: the threshold rule's sets, their order and the recorded
    margin follow from x alone (Th multi-select reading)."""
    rng = np.random.default_rng(14)
    n = 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    x = rng.standard_normal(n) * np.exp(rng.standard_normal(n))
    y = Q @ x
    th, k = 0.6, 9
    sets = _threshold_sets(x, th, k)
    o = oracle.clomp(Q, y, k, th=th, steps=30)
    assert o["support"][0].tolist() == [j for st in sets for j in st]
    assert int(o["n_iter"][0]) == k and int(o["status"][0]) == 0
    # margin of the first iteration, from x
    ax = np.abs(x)
    M = ax.max()
    first = sets[0]
    gaps = [(ax[j] - th * M) / M for j in first]
    gaps += [(ax[a] - ax[b]) / M for a, b in zip(first, first[1:])]
    gaps += [(th * M - ax[j]) / M for j in range(n) if j not in first and ax[j] < th * M]
    gaps += [(ax[first[-1]] - ax[j]) / M for j in range(n) if j not in first and ax[j] >= th * M]
    assert np.allclose(o["top1"][0, : len(first)] - o["top2"][0, : len(first)], min(gaps), atol=1e-12)


def test_clomp_threshold_room_caps_the_set():
    """More atoms pass than k allows: the largest ones are taken."""
    rng = np.random.default_rng(15)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    x = rng.standard_normal(n)
    o = oracle.clomp(Q, Q @ x, 3, th=1e-9, steps=10)
    assert o["support"][0].tolist() == np.argsort(-np.abs(x), kind="stable")[:3].tolist()
    assert int(o["n_iter"][0]) == 3 and int(o["status"][0]) == 0


def test_clomp_threshold_near_one_is_the_argmax_rule():
    """Th just below 1 keeps one atom per iteration on inputs without
    near-ties: the same support and coefficients as the argmax rule."""
    rng = np.random.default_rng(16)
    A = _rand_A(rng, 40, 120)
    Y = rng.standard_normal((40, 4))
    one = oracle.clomp(A, Y, 8, steps=20)
    thr = oracle.clomp(A, Y, 8, steps=20, th=1.0 - 1e-9)
    assert np.array_equal(one["support"], thr["support"])
    assert np.array_equal(one["coef"], thr["coef"])


# ---------------------------------------------------------------------------
# Column-wise 2D output path: x = D s, PSNR, SSIM (oracle/image.py)

def test_image_synthesize_orthonormal_round_trip():
    """Orthonormal DCT basis: the full code s = D^T x synthesises x back, in
    any support order, and entries past n_iter or < 0 are ignored."""
    from oracle import image as oi
    N = 64
    D = workloads.dct_synthesis(N)
    rng = np.random.default_rng(90)
    x = rng.standard_normal((N, 3))
    s = D.T @ x
    perm = [np.arange(N), rng.permutation(N), rng.permutation(N)]
    support = np.stack([p for p in perm])
    coef = np.stack([s[perm[b], b] for b in range(3)])
    X = oi.synthesize(D, support, coef, [N, N, N])
    np.testing.assert_allclose(X, x, atol=1e-12)
    sup2 = support.copy()
    sup2[1, 5] = -1
    X2 = oi.synthesize(D, sup2, coef, [N, 10, 0])
    np.testing.assert_allclose(X2[:, 1], D[:, support[1, :10]] @ coef[1, :10] - D[:, support[1, 5]] * coef[1, 5],
                               atol=1e-12)
    assert np.all(X2[:, 2] == 0.0)


def test_psnr_closed_form():
    from oracle import image as oi
    rng = np.random.default_rng(91)
    ref = rng.uniform(-2.0, 3.0, size=(40, 33))
    L = ref.max() - ref.min()
    # a constant offset d gives MSE = d^2
    assert abs(oi.psnr(ref + 0.03, ref) - 10.0 * np.log10(L * L / 0.03 ** 2)) < 1e-9
    assert abs(oi.psnr(ref - 0.5, ref, L=255.0) - 10.0 * np.log10(255.0 ** 2 / 0.25)) < 1e-9
    assert oi.psnr(ref, ref) == np.inf


def test_ssim_identity_symmetry_and_constant_images():
    from oracle import image as oi
    rng = np.random.default_rng(92)
    x = rng.standard_normal((30, 26))
    y = x + 0.3 * rng.standard_normal((30, 26))
    assert abs(oi.ssim(x, x) - 1.0) < 1e-14
    assert abs(oi.ssim(x, y, L=4.0) - oi.ssim(y, x, L=4.0)) < 1e-14
    assert oi.ssim(x, y) < 1.0
    # two constant images a, b: every window has zero variance, so the index
    # is the luminance term alone, (2ab + C1) / (a^2 + b^2 + C1)
    a, b, L = 0.7, 1.9, 2.0
    C1 = (0.01 * L) ** 2
    got = oi.ssim(np.full((16, 20), a), np.full((16, 20), b), L=L)
    # (the variances cancel to rounding: ~121 terms x 2^-52 x b^2 / C2 ~ 3e-11)
    assert abs(got - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-10


def test_ssim_against_window_by_window_loop():
    """The vectorised index equals a loop over every window placement with
    the weighted mean, centred variances and covariance written out."""
    from oracle import image as oi
    rng = np.random.default_rng(93)
    x = rng.uniform(0, 1, size=(14, 13))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    w = oi.gaussian_window()
    L = 1.0
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for i in range(14 - 11 + 1):
        for j in range(13 - 11 + 1):
            px, py = x[i:i + 11, j:j + 11], y[i:i + 11, j:j + 11]
            mx, my = (w * px).sum(), (w * py).sum()
            vx = (w * (px - mx) ** 2).sum()
            vy = (w * (py - my) ** 2).sum()
            cxy = (w * (px - mx) * (py - my)).sum()
            vals.append(((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2)))
    assert abs(oi.ssim(x, y, L=L) - np.mean(vals)) < 1e-13
    # the window is the 11 x 11 Gaussian of standard deviation 1.5, unit sum
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    assert abs(w[5, 5] / w[5, 6] - np.exp(1.0 / (2 * 1.5 ** 2))) < 1e-12


# ---------------------------------------------------------------------------
# Total-variation prior of Eq. 5 in the CL fit (oracle.tv_loss_grad, clomp(tv_weight))

def test_tv_value_and_gradient_closed_forms():
    """x = s (no basis): a ramp of slope c has TV = (n-1) c^2 / n; the
    gradient of w TV is (2w/n) L s with L the path-graph Laplacian
    (1, 2, ..., 2, 1 on the diagonal, -1 beside it)."""
    n, c, w = 7, 0.75, 1.3
    val, g = oracle.tv_loss_grad(None, n, list(range(n)), c * np.arange(n), w)
    assert abs(val - w * (n - 1) * c * c / n) < 1e-14
    Lap = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    Lap[0, 0] = Lap[-1, -1] = 1.0
    rng = np.random.default_rng(110)
    s = rng.standard_normal(n)
    _, g = oracle.tv_loss_grad(None, n, list(range(n)), s, w)
    np.testing.assert_allclose(g, (2.0 * w / n) * (Lap @ s), atol=1e-14)
    # a subset support sees the Laplacian's rows and columns of its atoms
    S = [5, 1, 3]
    _, gS = oracle.tv_loss_grad(None, n, S, s[S], w)
    np.testing.assert_allclose(gS, (2.0 * w / n) * (Lap[np.ix_(S, S)] @ s[S]), atol=1e-14)


def test_tv_gradient_matches_central_differences():
    """The whole CL loss 1/2||y - A_S s||^2 + w TV(D_S s) is quadratic in s,
    so central differences are exact up to rounding."""
    rng = np.random.default_rng(111)
    m, n, N, w = 9, 10, 14, 0.8
    A = rng.standard_normal((m, n))
    D = rng.standard_normal((N, n))
    y = rng.standard_normal(m)
    S = np.array([7, 2, 9, 4], dtype=np.int32)
    s = rng.standard_normal(4)

    def loss(v):
        r = y - A[:, S] @ v
        x = D[:, S] @ v
        return 0.5 * r @ r + w * np.sum(np.diff(x) ** 2) / N

    _, g_data, _ = oracle.clfit_loss_grad(A, S, s, y)
    _, g_tv = oracle.tv_loss_grad(D, n, S, s, w)
    h = 1e-4
    fd = np.array([(loss(s + h * e) - loss(s - h * e)) / (2 * h) for e in np.eye(4)])
    np.testing.assert_allclose(g_data + g_tv, fd, rtol=1e-8, atol=1e-9)


def test_clomp_with_tv_prior_is_adam_on_the_prior_loss():
    """CLOMP with the prior: one torch Adam run (float64, autograd) on
    1/2||y - A(p * mask)||^2 + w TV(D (p * mask)), T steps per pick, the
    mask growing by the picks of the residual's correlation."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(112)
    m, n, N, k, T, w = 20, 40, 40, 4, 25, 0.6
    A = _rand_A(rng, m, n)
    D = workloads.dct_synthesis(N)
    y = rng.standard_normal(m)
    o = oracle.clomp(A, y, k, steps=T, lr=3e-2, tv_weight=w, D=D)
    S = o["support"][0]
    p = torch.zeros(n, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-2, foreach=False)
    At = torch.tensor(A, dtype=torch.float64)
    Dt = torch.tensor(D, dtype=torch.float64)
    yt = torch.tensor(y, dtype=torch.float64)
    mask = torch.zeros(n, dtype=torch.float64)
    for t in range(k):
        r = (yt - At @ (p * mask)).detach()
        c = (At.T @ r).abs().numpy()
        c[mask.numpy() > 0] = -1
        assert int(np.argmax(c)) == S[t]
        mask[S[t]] = 1.0
        for _ in range(T):
            opt.zero_grad()
            v = p * mask
            x = Dt @ v
            loss = 0.5 * torch.sum((yt - At @ v) ** 2) + w * torch.sum((x[1:] - x[:-1]) ** 2) / N
            loss.backward()
            opt.step()
    np.testing.assert_allclose(o["coef"][0], p.detach().numpy()[S], rtol=0, atol=1e-12)
    # w = 0 is the plain CLOMP
    o0 = oracle.clomp(A, y, k, steps=T, lr=3e-2, tv_weight=0.0, D=D)
    o1 = oracle.clomp(A, y, k, steps=T, lr=3e-2)
    assert np.array_equal(o0["coef"], o1["coef"]) and np.array_equal(o0["support"], o1["support"])


# Total variation of an image (Eq. 6) in the CL fit: oracle.tv2d_h_loss_grad
# (the horizontal part) and clomp(image_width=W), which fits the W columns of an
# image together

def test_tv2d_horizontal_closed_forms():
    """x_j = s_j (no basis), every pixel of column j equal to c j: each of the
    W - 1 neighbouring pairs differs by c in all n pixels, so TV_h =
    (W - 1) n c^2 / W; alternating columns +-c differ by 2c.  Columns with
    disjoint supports see each other's coefficients as zeros."""
    n, W, c, w = 6, 5, 0.5, 1.7
    full = list(range(n))
    val, g = oracle.tv2d_h_loss_grad(None, n, [full] * W, [c * j * np.ones(n) for j in range(W)], w)
    assert abs(val - w * (W - 1) * n * c * c / W) < 1e-13
    # interior columns of a ramp have zero gradient; the ends are pulled inwards
    for j in range(1, W - 1):
        np.testing.assert_allclose(g[j], 0.0, atol=1e-14)
    np.testing.assert_allclose(g[0], -2.0 * w * c / W, rtol=1e-14)
    np.testing.assert_allclose(g[-1], 2.0 * w * c / W, rtol=1e-14)
    val, _ = oracle.tv2d_h_loss_grad(None, n, [full] * W, [c * (-1) ** j * np.ones(n) for j in range(W)], w)
    assert abs(val - w * (W - 1) * n * 4 * c * c / W) < 1e-13
    val, g = oracle.tv2d_h_loss_grad(None, n, [[0, 1], [2, 3]], [np.array([1.0, 2.0]), np.array([3.0, -1.0])], w)
    assert abs(val - w * (1 + 4 + 9 + 1) / 2) < 1e-14
    np.testing.assert_allclose(g[0], w * np.array([1.0, 2.0]), rtol=1e-14)
    np.testing.assert_allclose(g[1], w * np.array([3.0, -1.0]), rtol=1e-14)
    # one column: no horizontal pairs
    assert oracle.tv2d_h_loss_grad(None, n, [full], [np.ones(n)], w)[0] == 0.0


def test_tv2d_gradient_matches_central_differences():
    """Image loss sum_j 1/2||y_j - A_Sj s_j||^2 + w TV(I), I = [D s_1 .. D s_W]
    (Eq. 6: (1/H) sum of vertical squared differences + (1/W) sum of
    horizontal ones), a quadratic: central differences are exact up to
    rounding.  D is a general (non-orthonormal) basis."""
    rng = np.random.default_rng(150)
    m, n, H, W, w = 7, 9, 11, 4, 0.9
    A = rng.standard_normal((m, n))
    D = rng.standard_normal((H, n))
    Y = rng.standard_normal((m, W))
    sup = [np.array([3, 1, 8], np.int32), np.array([1, 5], np.int32), np.array([8, 3, 0, 6], np.int32),
           np.array([2], np.int32)]
    coefs = [rng.standard_normal(len(q)) for q in sup]

    def loss(cs):
        I = np.stack([D[:, q] @ v for q, v in zip(sup, cs)], axis=1)     # H x W image
        data = sum(0.5 * np.sum((Y[:, j] - A[:, q] @ v) ** 2) for j, (q, v) in enumerate(zip(sup, cs)))
        vert = np.sum((I[:-1, :] - I[1:, :]) ** 2) / H
        horiz = np.sum((I[:, :-1] - I[:, 1:]) ** 2) / W
        return data + w * (vert + horiz)

    _, gh = oracle.tv2d_h_loss_grad(D, n, sup, coefs, w)
    h = 1e-4
    for j in range(W):
        _, gd, _ = oracle.clfit_loss_grad(A, sup[j], coefs[j], Y[:, j])
        _, gv = oracle.tv_loss_grad(D, n, sup[j], coefs[j], w)
        fd = []
        for e in np.eye(len(sup[j])):
            up = [v.copy() for v in coefs]
            dn = [v.copy() for v in coefs]
            up[j] += h * e
            dn[j] -= h * e
            fd.append((loss(up) - loss(dn)) / (2 * h))
        np.testing.assert_allclose(gd + gv + gh[j], fd, rtol=1e-8, atol=1e-9)


def test_clomp_tv2d_is_adam_on_the_image_loss():
    """CLOMP with the image prior: one torch Adam run (float64, autograd) over
    the n x W learnable coefficients of an image, loss sum_j 1/2||y_j -
    A(p_j * mask_j)||^2 + w TV(D (P * Mask)) (Eq. 6), T steps per iteration,
    each column's mask growing by the pick of its own residual's
    correlation."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(151)
    m, n, W, k, T, w = 16, 32, 5, 4, 20, 0.7
    A = _rand_A(rng, m, n)
    D = workloads.dct_synthesis(n)
    Y = rng.standard_normal((m, W))
    o = oracle.clomp(A, Y, k, steps=T, lr=3e-2, tv_weight=w, D=D, image_width=W)
    assert np.all(o["status"] == 0) and np.all(o["n_iter"] == k)
    P = torch.zeros((n, W), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([P], lr=3e-2, foreach=False)
    At = torch.tensor(A, dtype=torch.float64)
    Dt = torch.tensor(D, dtype=torch.float64)
    Yt = torch.tensor(Y, dtype=torch.float64)
    mask = torch.zeros((n, W), dtype=torch.float64)
    for t in range(k):
        R = (Yt - At @ (P * mask)).detach()
        C = (At.T @ R).abs().numpy()
        C[mask.numpy() > 0] = -1
        for j in range(W):
            assert int(np.argmax(C[:, j])) == o["support"][j, t]
            mask[o["support"][j, t], j] = 1.0
        for _ in range(T):
            opt.zero_grad()
            V = P * mask
            I = Dt @ V
            loss = (0.5 * torch.sum((Yt - At @ V) ** 2)
                    + w * (torch.sum((I[1:, :] - I[:-1, :]) ** 2) / n + torch.sum((I[:, 1:] - I[:, :-1]) ** 2) / W))
            loss.backward()
            opt.step()
    Pn = P.detach().numpy()
    for j in range(W):
        np.testing.assert_allclose(o["coef"][j], Pn[o["support"][j], j], rtol=0, atol=1e-12)


def test_clomp_tv2d_reductions():
    """Identical columns stay identical, so the horizontal term vanishes and
    the image fit is the per-column fit with the 1-D prior; one-column images
    have no horizontal pairs; w = 0 is plain CLOMP."""
    rng = np.random.default_rng(152)
    m, n, k = 24, 48, 5
    A = _rand_A(rng, m, n)
    D = workloads.dct_synthesis(n)
    y = rng.standard_normal(m)
    Y = np.repeat(y[:, None], 6, axis=1)
    a = oracle.clomp(A, Y, k, steps=30, tv_weight=0.8, D=D, image_width=3)
    b = oracle.clomp(A, Y, k, steps=30, tv_weight=0.8, D=D)
    assert np.array_equal(a["support"], b["support"])
    np.testing.assert_allclose(a["coef"], b["coef"], rtol=0, atol=1e-15)
    Y2 = rng.standard_normal((m, 4))
    a = oracle.clomp(A, Y2, k, steps=30, tv_weight=0.8, D=D, image_width=1)
    b = oracle.clomp(A, Y2, k, steps=30, tv_weight=0.8, D=D)
    assert np.array_equal(a["support"], b["support"]) and np.array_equal(a["coef"], b["coef"])
    a = oracle.clomp(A, Y2, k, steps=30, tv_weight=0.0, D=D, image_width=2)
    b = oracle.clomp(A, Y2, k, steps=30)
    assert np.array_equal(a["support"], b["support"]) and np.array_equal(a["coef"], b["coef"])


# Local variation of Eq. 7 (oracle.lv_loss_grad, clomp(lv_weight, image_width))

def test_lv_closed_forms():
    """3 x 3 windows at every placement, sample standard deviation: a ramp of
    step c along either axis puts {0, c, 2c} three times in every window, so
    each window's deviation is c sqrt(6/8) and so is their mean; a constant
    image has LV = 0 and zero gradient; a single 3 x 3 image is the sample
    standard deviation of its nine pixels (numpy, ddof=1)."""
    n, W, c, w = 7, 6, 0.4, 1.9
    full = list(range(n))
    val, g = oracle.lv_loss_grad(None, n, [full] * W, [c * j * np.ones(n) for j in range(W)], w)
    assert abs(val - w * c * math.sqrt(0.75)) < 1e-14
    val, _ = oracle.lv_loss_grad(None, n, [full] * W, [c * np.arange(n) for _ in range(W)], w)
    assert abs(val - w * c * math.sqrt(0.75)) < 1e-14
    val, g = oracle.lv_loss_grad(None, n, [full] * W, [2.5 * np.ones(n) for _ in range(W)], w)
    assert val == 0.0 and all(np.all(q == 0.0) for q in g)
    rng = np.random.default_rng(180)
    v = rng.standard_normal((3, 3))
    val, _ = oracle.lv_loss_grad(None, 3, [[0, 1, 2]] * 3, [v[:, j] for j in range(3)], 1.0)
    assert abs(val - np.std(v, ddof=1)) < 1e-14
    # fewer than three rows or columns: no window
    assert oracle.lv_loss_grad(None, n, [full] * 2, [np.ones(n), -np.ones(n)], w)[0] == 0.0


def test_lv_gradient_matches_central_differences():
    """LV is smooth where no window is constant: central differences of
    w LV(I), I = [D s_1 .. D s_W] with a general basis, to 1e-7."""
    rng = np.random.default_rng(181)
    n, H, W, w = 9, 8, 5, 1.3
    D = rng.standard_normal((H, n))
    sup = [np.array([3, 1, 8], np.int32), np.array([1, 5], np.int32), np.array([8, 3, 0, 6], np.int32),
           np.array([2], np.int32), np.array([7, 4], np.int32)]
    coefs = [rng.standard_normal(len(q)) for q in sup]

    def lv(cs):
        I = np.stack([D[:, q] @ v for q, v in zip(sup, cs)], axis=1)
        sig = [np.std(I[r:r + 3, c:c + 3], ddof=1) for r in range(H - 2) for c in range(W - 2)]
        return w * np.mean(sig)

    val, g = oracle.lv_loss_grad(D, n, sup, coefs, w)
    assert abs(val - lv(coefs)) < 1e-13
    h = 1e-5
    for j in range(W):
        fd = []
        for e in np.eye(len(sup[j])):
            up = [v.copy() for v in coefs]
            dn = [v.copy() for v in coefs]
            up[j] += h * e
            dn[j] -= h * e
            fd.append((lv(up) - lv(dn)) / (2 * h))
        np.testing.assert_allclose(g[j], fd, rtol=1e-6, atol=1e-9)


def test_clomp_lv_is_adam_on_the_image_loss():
    """CLOMP with both image priors: one torch Adam run (float64, autograd)
    over the n x W coefficients, loss data + w_tv TV(I) + w_lv LV(I); a
    constant window (all pixels zero at the start) contributes no gradient."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(182)
    m, n, W, k, T, wt, wl = 16, 32, 6, 4, 20, 0.4, 0.9
    A = _rand_A(rng, m, n)
    D = workloads.dct_synthesis(n)
    Y = rng.standard_normal((m, W))
    o = oracle.clomp(A, Y, k, steps=T, lr=3e-2, tv_weight=wt, lv_weight=wl, D=D, image_width=W)
    assert np.all(o["status"] == 0) and np.all(o["n_iter"] == k)
    P = torch.zeros((n, W), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([P], lr=3e-2, foreach=False)
    At = torch.tensor(A, dtype=torch.float64)
    Dt = torch.tensor(D, dtype=torch.float64)
    Yt = torch.tensor(Y, dtype=torch.float64)
    mask = torch.zeros((n, W), dtype=torch.float64)

    def lv(I):
        win = I.unfold(0, 3, 1).unfold(1, 3, 1).reshape(-1, 9)       # every 3 x 3 placement
        var = torch.sum((win - win.mean(dim=1, keepdim=True)) ** 2, dim=1) / 8.0
        sig = torch.where(var > 0, torch.sqrt(torch.clamp(var, min=1e-300)), torch.zeros_like(var))
        return sig.mean()

    for t in range(k):
        R = (Yt - At @ (P * mask)).detach()
        C = (At.T @ R).abs().numpy()
        C[mask.numpy() > 0] = -1
        for j in range(W):
            assert int(np.argmax(C[:, j])) == o["support"][j, t]
            mask[o["support"][j, t], j] = 1.0
        for _ in range(T):
            opt.zero_grad()
            V = P * mask
            I = Dt @ V
            tv = torch.sum((I[1:, :] - I[:-1, :]) ** 2) / n + torch.sum((I[:, 1:] - I[:, :-1]) ** 2) / W
            loss = 0.5 * torch.sum((Yt - At @ V) ** 2) + wt * tv + wl * lv(I)
            loss.backward()
            opt.step()
    Pn = P.detach().numpy()
    for j in range(W):
        np.testing.assert_allclose(o["coef"][j], Pn[o["support"][j], j], rtol=0, atol=1e-12)
    # w_lv = 0 is the image TV alone
    a = oracle.clomp(A, Y, k, steps=T, lr=3e-2, tv_weight=wt, lv_weight=0.0, D=D, image_width=W)
    b = oracle.clomp(A, Y, k, steps=T, lr=3e-2, tv_weight=wt, D=D, image_width=W)
    assert np.array_equal(a["coef"], b["coef"])


def test_lv_smoothed_deviation():
    """sqrt(var + eps^2): a constant image gives LV = eps with zero gradient, a
    ramp sqrt(0.75 c^2 + eps^2); the smoothed loss is differentiable at
    constant windows, so central differences hold on a mostly-zero image
    (x = s, many constant windows); and a torch Adam run with the smoothed
    deviation reproduces the image fit."""
    n, W, c, w, eps = 7, 6, 0.4, 1.9, 0.05
    full = list(range(n))
    val, g = oracle.lv_loss_grad(None, n, [full] * W, [2.5 * np.ones(n) for _ in range(W)], w, eps)
    assert abs(val - w * eps) < 1e-15 and all(np.all(q == 0.0) for q in g)
    val, _ = oracle.lv_loss_grad(None, n, [full] * W, [c * j * np.ones(n) for j in range(W)], w, eps)
    assert abs(val - w * math.sqrt(0.75 * c * c + eps * eps)) < 1e-14
    rng = np.random.default_rng(190)
    n, W = 20, 7
    sup = [rng.choice(n, 2, replace=False).astype(np.int32) for _ in range(W)]
    coefs = [rng.standard_normal(2) for _ in range(W)]

    def lv(cs):
        I = np.zeros((n, W))
        for j, (q, v) in enumerate(zip(sup, cs)):
            I[q, j] += v
        sig = [math.sqrt(np.var(I[r:r + 3, cc:cc + 3], ddof=1) + eps * eps)
               for r in range(n - 2) for cc in range(W - 2)]
        return w * np.mean(sig)

    val, g = oracle.lv_loss_grad(None, n, sup, coefs, w, eps)
    assert abs(val - lv(coefs)) < 1e-13
    h = 1e-6
    for j in range(W):
        fd = []
        for e in np.eye(2):
            up = [v.copy() for v in coefs]
            dn = [v.copy() for v in coefs]
            up[j] += h * e
            dn[j] -= h * e
            fd.append((lv(up) - lv(dn)) / (2 * h))
        np.testing.assert_allclose(g[j], fd, rtol=1e-6, atol=1e-10)
    torch = pytest.importorskip("torch")
    m, n, W, k, T, wl = 16, 32, 5, 3, 20, 0.9
    A = _rand_A(rng, m, n)
    D = workloads.dct_synthesis(n)
    Y = rng.standard_normal((m, W))
    o = oracle.clomp(A, Y, k, steps=T, lr=3e-2, lv_weight=wl, lv_eps=eps, D=D, image_width=W)
    P = torch.zeros((n, W), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([P], lr=3e-2, foreach=False)
    At, Dt, Yt = (torch.tensor(v, dtype=torch.float64) for v in (A, D, Y))
    mask = torch.zeros((n, W), dtype=torch.float64)
    for t in range(k):
        for j in range(W):
            mask[o["support"][j, t], j] = 1.0
        for _ in range(T):
            opt.zero_grad()
            V = P * mask
            win = (Dt @ V).unfold(0, 3, 1).unfold(1, 3, 1).reshape(-1, 9)
            var = torch.sum((win - win.mean(dim=1, keepdim=True)) ** 2, dim=1) / 8.0
            loss = 0.5 * torch.sum((Yt - At @ V) ** 2) + wl * torch.sqrt(var + eps * eps).mean()
            loss.backward()
            opt.step()
    Pn = P.detach().numpy()
    for j in range(W):
        np.testing.assert_allclose(o["coef"][j], Pn[o["support"][j], j], rtol=0, atol=1e-12)


def test_clomp_image_stopped_column_is_frozen_neighbour():
    """An image whose second column is one atom exactly stops after its first
    iteration (tol); the other columns go on, and the stopped column keeps its
    coefficient yet still pulls on its neighbours through the horizontal TV.
    Torch reference: one float64 Adam per column (its own state and step
    counter), a column steps only while it is live."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(195)
    m, n, W, k, T, lr, w, tol = 16, 32, 4, 4, 100, 5e-2, 0.4, 0.8
    A = rng.standard_normal((m, n))
    A /= np.linalg.norm(A, axis=0)
    D = workloads.dct_synthesis(n)
    Y = rng.standard_normal((m, W))
    Y[:, 1] = 2.0 * A[:, 5]
    Y[:, 2] += 3.0 * A[:, 5]          # the third column picks atom 5 too
    o = oracle.clomp(A, Y, k, tol=tol, steps=T, lr=lr, tv_weight=w, D=D, image_width=W)
    assert list(o["n_iter"]) == [4, 1, 4, 4] and list(o["status"]) == [0, 1, 0, 0]
    assert o["support"][2, 0] == 5
    At, Dt, Yt = (torch.tensor(v, dtype=torch.float64) for v in (A, D, Y))
    P = [torch.zeros(n, dtype=torch.float64, requires_grad=True) for _ in range(W)]
    opts = [torch.optim.Adam([p], lr=lr, foreach=False) for p in P]
    mask = torch.zeros((n, W), dtype=torch.float64)
    live = [True] * W
    for t in range(k):
        for j in range(W):
            if live[j]:
                r = (Yt[:, j] - At @ (P[j] * mask[:, j])).detach()
                c = (At.T @ r).abs().numpy()
                c[mask[:, j].numpy() > 0] = -1
                a = int(np.argmax(c))
                assert a == o["support"][j, t]
                mask[a, j] = 1.0
        for _ in range(T):
            for opt in opts:
                opt.zero_grad()
            V = torch.stack(P, dim=1) * mask
            I = Dt @ V
            loss = (0.5 * torch.sum((Yt - At @ V) ** 2)
                    + w * (torch.sum((I[1:, :] - I[:-1, :]) ** 2) / n + torch.sum((I[:, 1:] - I[:, :-1]) ** 2) / W))
            loss.backward()
            for j in range(W):
                if live[j]:
                    opts[j].step()
        for j in range(W):
            if live[j]:
                res = float(torch.linalg.norm(Yt[:, j] - At @ (P[j].detach() * mask[:, j])))
                if res <= tol:
                    live[j] = False
    for j in range(W):
        np.testing.assert_allclose(o["coef"][j, :o["n_iter"][j]], P[j].detach().numpy()[o["support"][j, :o["n_iter"][j]]],
                                   rtol=0, atol=1e-12)
    # the frozen column still pulls its neighbour's coefficient of their
    # shared atom: with the column zero (stopped at once, s = 0) it differs
    Y0 = Y.copy()
    Y0[:, 1] = 0.0
    o0 = oracle.clomp(A, Y0, k, tol=tol, steps=T, lr=lr, tv_weight=w, D=D, image_width=W)
    assert o0["n_iter"][1] == 0 and o0["support"][2, 0] == 5
    assert abs(o0["coef"][2, 0] - o["coef"][2, 0]) > 1e-3


# ---------------------------------------------------------------- IHT pins
def test_iht_orthonormal_closed_form():
    """A orthonormal (m = n), t = 1: the first iteration gives
    s = H_k(A^T y) and every later one returns the same point; ||r||^2 =
    ||y||^2 - the kept sum of (A^T y)_j^2."""
    rng = np.random.default_rng(41)
    n, k = 24, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Y = rng.standard_normal((n, 3))
    for it in (1, 4):
        o = oracle.iht(Q, Y, k, 1.0, max_iter=it)
        for b in range(3):
            c = Q.T @ Y[:, b]
            keep = np.sort(np.argsort(-np.abs(c), kind="stable")[:k])
            assert o["support"][b].tolist() == keep.tolist()
            assert np.allclose(o["coef"][b], c[keep], atol=1e-12)
            assert abs(o["res_norm"][b] ** 2 - (np.sum(Y[:, b] ** 2) - np.sum(c[keep] ** 2))) < 1e-10
            assert o["n_iter"][b] == it and o["status"][b] == 2


def test_iht_ties_keep_the_lowest_indices():
    y = np.array([1.0, -1.0, 1.0, 0.5, -1.0, 0.2])
    o = oracle.iht(np.eye(6), y, 3, 1.0, max_iter=1)
    assert o["support"][0].tolist() == [0, 1, 2]
    assert o["coef"][0].tolist() == [1.0, -1.0, 1.0]
    assert o["margin"][0] == 0.0


def test_iht_objective_non_increasing_for_small_steps():
    """With t <= 1 / sigma_max(A)^2 the residual norm of IHT does not grow
    (Blumensath and Davies, 2008)."""
    rng = np.random.default_rng(42)
    A = _rand_A(rng, 40, 120)
    Y = workloads.add_noise(rng, A @ workloads.sparse_coefficients(rng, 120, 4, 6), 20.0)
    t = 0.99 / np.linalg.norm(A, 2) ** 2
    prev = np.full(4, np.inf)
    for it in range(1, 31):
        o = oracle.iht(A, Y, 6, t, max_iter=it)
        assert np.all(o["res_norm"] <= prev * (1 + 1e-12))
        prev = o["res_norm"]


def test_iht_noiseless_recovery():
    """Noiseless sparse signals that IHT recovers (residual at rounding
    level) come back with their exact support and coefficients; most of
    them are recovered."""
    rng = np.random.default_rng(43)
    A = _rand_A(rng, 120, 300)
    X = workloads.sparse_coefficients(rng, 300, 8, 6)
    Y = A @ X
    o = oracle.iht(A, Y, 6, 1.0 / np.linalg.norm(A, 2) ** 2, max_iter=3000)
    ok = o["res_norm"] <= 1e-9 * np.linalg.norm(Y, axis=0)
    assert ok.sum() >= 6
    for b in np.nonzero(ok)[0]:
        assert o["support"][b].tolist() == np.nonzero(X[:, b])[0].tolist()
        assert np.allclose(o["coef"][b], X[o["support"][b], b], atol=1e-8)


def test_iht_keeping_everything_is_landweber():
    """k = n: H_k keeps every entry and IHT is gradient descent on
    1/2 ||y - A s||^2, which converges to the least-squares solution of a
    full-column-rank A (numpy lstsq, library)."""
    rng = np.random.default_rng(44)
    A = rng.standard_normal((30, 10))
    y = rng.standard_normal(30)
    o = oracle.iht(A, y, 10, 1.0 / np.linalg.norm(A, 2) ** 2, max_iter=4000)
    assert o["support"][0].tolist() == list(range(10))
    assert np.allclose(o["coef"][0], np.linalg.lstsq(A, y, rcond=None)[0], atol=1e-9)
    assert o["margin"][0] == 1.0


def test_iht_stop_rules():
    rng = np.random.default_rng(45)
    A = _rand_A(rng, 16, 40)
    Y = rng.standard_normal((16, 3))
    Y[3, 1] = np.nan
    Y[:, 2] = 0.0
    o = oracle.iht(A, Y, 4, 0.2, tol=1e-9, max_iter=7)
    assert o["status"].tolist() == [2, 4, 1]
    assert o["n_iter"].tolist() == [7, 0, 0]
    assert np.all(o["support"][1] == -1) and np.all(o["support"][2] == -1)
    z = A[:, [3, 11]] @ np.array([2.0, -1.0])
    o = oracle.iht(np.eye(16), z[:16], 16, 1.0, tol=1e-12, max_iter=50)
    assert o["status"][0] == 1 and o["n_iter"][0] == 1
