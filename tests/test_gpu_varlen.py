"""Uneven batches (instances of different n, m, k with their own A) through
the varlen C-ABI entry points, against the FP64 oracle per instance, at the
batch's stated sizes."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from parity import compare, f32

pytestmark = pytest.mark.gpu


def test_varlen_refuses_instances_beyond_the_plan(cs_gpu):
    """An instance larger than the plan is not solved (status UNSUPPORTED,
    support -1, coef 0, n_iter 0, res_norm ||y||); the others still are."""
    import torch
    p = workloads.random_problem(16, 100, 2, 4, seed=3, snr_db=30.0)
    A_small = torch.from_numpy(np.asfortranarray(p.A, dtype=np.float32)).cuda()
    A_big = torch.randn(32, 100, device="cuda")
    y_big = torch.randn(32, device="cuda")
    plan = cs_gpu.Plan(16, 100, 8, 8)
    ys = [torch.from_numpy(np.float32(p.Y[:, b])).cuda() for b in range(2)]
    outs = cs_gpu.omp_solve_varlen([(A_small, ys[0], 4), (A_big, y_big, 4), (A_small, ys[1], 4)], plan=plan)
    torch.cuda.synchronize()
    o = outs[1]
    assert int(o.status[0]) == cs_gpu.SIG_UNSUPPORTED and int(o.n_iter[0]) == 0
    assert (o.support == -1).all() and (o.coef == 0).all()
    assert abs(float(o.res_norm[0]) - float(torch.linalg.norm(y_big))) <= 1e-5 * float(torch.linalg.norm(y_big))
    for b in (0, 2):
        assert int(outs[b].status[0]) == cs_gpu.SIG_REACHED_K and int(outs[b].n_iter[0]) == 4


def test_varlen_rejects_malformed_instances(cs_gpu):
    import torch
    A = torch.randn(8, 100, device="cuda")
    y = torch.randn(8, device="cuda")
    plan = cs_gpu.Plan(16, 100, 8, 16)
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.omp_solve_varlen([(A, y, 9)], plan=plan)      # k > m
    assert e.value.code == -1


# The plan of the stated-size uneven batch below, and the limits the header
# documents for a solved instance: OMP and CLOMP (Gram form) solve every
# instance within the plan, beyond the on-chip kernels on the large-instance
# path.
_C5_PLAN = (8192, 16384, 128, 2048)


def _c5_solvable(m, n, k, prec, algo):
    m_max, n_max, _, k_max = _C5_PLAN
    return m <= m_max and n <= n_max and k <= k_max


def _on_chip(m, n, k, prec):
    return m <= 1024 and k <= 64 and (prec == "fp32" or (m <= 256 and n <= 4096))


_C5_ORACLE = {}


@pytest.mark.parametrize("algo,prec", [("omp", "fp32"), ("omp", "bf16"), ("clomp", "bf16")])
def test_uneven_batch_at_stated_sizes(cs_gpu, algo, prec):
    """The uneven batch as stated (2000 instances, n log-uniform in
    [512, 16384], m/n in [0.1, 0.5], k = 1-10 % of n, Gaussian or Bernoulli A,
    30 dB): every instance within the documented limits is solved, every
    other one is refused with CS_SIG_UNSUPPORTED.  Solved instances of the
    on-chip kernels are all compared with the FP64 oracle; of those on the
    large-instance path, the one with the least oracle work in each size
    class (oracle runs of the others would take hours), excluding the
    ill-conditioned k > m / 2 ones whose float32 Gram matrices decide the
    coefficients (their count is printed).  The refused instances' A is never
    read, so classes without a solvable instance are not materialised."""
    import concurrent.futures as cf
    import torch
    classes, assign, ks = workloads.config_uneven()
    solvable = [_c5_solvable(classes[assign[i]]["m"], classes[assign[i]]["n"], ks[i], prec, algo)
                for i in range(len(assign))]
    dummy_A = torch.zeros(1, device="cuda")
    keep, data = [dummy_A], {}
    arr = (cs_gpu.Instance * len(assign))()
    outs = [cs_gpu._outputs(1, ks[i], "cuda") for i in range(len(assign))]
    rng = np.random.default_rng(5)

    def put(i, A_ptr, m, n, y):
        o = outs[i]
        arr[i] = cs_gpu.Instance(A_ptr, m, n, m, y.data_ptr(), ks[i], o.support.data_ptr(), o.coef.data_ptr(),
                                 o.n_iter.data_ptr(), o.res_norm.data_ptr(), o.status.data_ptr())
        keep.append(y)

    for c, cl in enumerate(classes):
        idx = [i for i in range(len(assign)) if assign[i] == c]
        if any(solvable[i] for i in idx):
            A, inst = workloads.uneven_class_data(classes, assign, ks, c, dtype=np.float32)
            At = torch.from_numpy(A).cuda()
            keep.append(At)
            for i, y, _ in inst:
                put(i, At.data_ptr(), cl["m"], cl["n"], torch.from_numpy(np.float32(y)).cuda())
                data[i] = (A, np.float32(y))
        else:
            # refused whole classes: their A is never read, so it is not drawn
            for i in idx:
                put(i, dummy_A.data_ptr(), cl["m"], cl["n"],
                    torch.from_numpy(rng.standard_normal(cl["m"]).astype(np.float32)).cuda())
    plan = cs_gpu.Plan(*_C5_PLAN)
    L = cs_gpu.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if algo == "omp":
        prm = cs_gpu._omp_params(1, 0.0, 0, prec, 0)
        rc = L.omp_solve_varlen(plan.h, arr, len(assign), ctypes.byref(prm), stream)
    else:
        prm = cs_gpu._clomp_params(1, 0.0, 0, prec, 0, 50, 1e-2, 0.9, 0.999, 1e-8, False, "gram")
        rc = L.clomp_solve_varlen(plan.h, arr, len(assign), ctypes.byref(prm), stream)
    assert rc == 0, L.cs_last_error()
    torch.cuda.synchronize()
    status = np.array([int(o.status[0]) for o in outs])
    assert np.all((status == cs_gpu.SIG_UNSUPPORTED) == ~np.array(solvable)), "refusals differ from the limits"
    for i in np.nonzero(~np.array(solvable))[0]:
        o = outs[i]
        assert int(o.n_iter[0]) == 0 and bool((o.support == -1).all())
    okw = dict(lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))

    def reference(i):
        key = (algo, i)
        if key not in _C5_ORACLE:
            A, y = data[i]
            A64, y64 = A.astype(np.float64), y.astype(np.float64)
            _C5_ORACLE[key] = (oracle.omp(A64, y64, ks[i], nthreads=1) if algo == "omp"
                               else oracle.clomp(A64, y64, ks[i], steps=50, nthreads=1, **okw))
        return _C5_ORACLE[key]

    def check(i):
        o = outs[i]
        g = {q: getattr(o, q).cpu().numpy() for q in ("support", "coef", "n_iter", "res_norm", "status")}
        return compare(g, reference(i), check_status=True)

    dims = lambda i: (classes[assign[i]]["m"], classes[assign[i]]["n"], ks[i])
    solved = [i for i in range(len(assign)) if solvable[i]]
    chip = [i for i in solved if _on_chip(*dims(i), prec)]
    large = [i for i in solved if not _on_chip(*dims(i), prec)]
    ill = [i for i in large if dims(i)[2] > dims(i)[0] / 2]
    sample = {}
    for i in large:
        m, n, k = dims(i)
        if k > m / 2:
            continue
        c = assign[i]
        if c not in sample or k * m * n < np.prod(dims(sample[c])):
            sample[c] = i
    todo = chip + sorted(sample.values())
    # every solved instance: a valid support of distinct atoms, k of them unless stopped early
    for i in solved:
        o = outs[i]
        m, n, k = dims(i)
        t, st = int(o.n_iter[0]), int(o.status[0])
        sup = o.support[0].cpu().numpy()
        assert st in (0, 1, 2, 3) and 0 <= t <= k and (st != 0 or t == k), (i, st, t, k)
        assert len(set(sup[:t].tolist())) == t and np.all((sup[:t] >= 0) & (sup[:t] < n)) and np.all(sup[t:] == -1)
    with cf.ThreadPoolExecutor(max_workers=max(1, oracle.max_threads())) as ex:
        summaries = list(ex.map(check, todo))
    ambiguous = sum(s["ambiguous"] for s in summaries)
    assert ambiguous <= max(1, len(todo) // 100)
    _, errs = plan.counters(reset=True)
    assert errs == 0
    print(f"uneven batch ({algo}, {prec}): {len(solved)} of {len(assign)} instances solved "
          f"({len(chip)} on chip, {len(large)} on the large path, {len(ill)} of them with k > m/2), "
          f"{len(todo)} compared with the oracle, {len(assign) - len(solved)} refused, {ambiguous} ambiguous")
