"""A kept as a fixed layer across solves (cs_plan_set_A_generation): solves
that reuse A's preparation give bit-identical results to solves that prepare
A again, skip exactly the preparation launches, and a new generation (or the
TV prior, which changes A^T A in place) makes the next solve prepare A."""
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


def setup_launches(plan):
    return plan.profile(reset=True)["setup"][0]


def run(cs, torch, plan, A, Y, k, algo, prec, **kw):
    if algo == "omp":
        r = cs.omp_solve_batched(A, Y, k, prec=prec, plan=plan)
    else:
        r = cs.clomp_solve_batched(A, Y, k, prec=prec, plan=plan, form="gram", **CL, **kw)
    torch.cuda.synchronize()
    assert plan.counters()[1] == 0
    return to_numpy(r)


def same(a, b):
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(a[q], b[q]), q


@pytest.mark.parametrize("algo,prec,graphs", [("clomp", "bf16", 0), ("clomp", "bf16", 1),
                                              ("clomp", "fp32", 0), ("omp", "fp32", 0),
                                              ("omp", "bf16", 0)])
def test_reuse_matches_fresh_preparation(cs_gpu, torch, algo, prec, graphs):
    cs = cs_gpu
    m, n, B, k = 64, 256, 320, 8
    p1 = workloads.random_problem(m, n, B, k, seed=141, snr_db=40.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p1.A, p1.Y)
    Y2 = np.asfortranarray(workloads.random_problem(m, n, B, k, seed=142, values="pm").Y, np.float32)
    A = torch.from_numpy(A32).cuda()
    Ya, Yb = torch.from_numpy(Y32).cuda(), torch.from_numpy(Y2).cuda()

    fresh = cs.Plan(m, n, B, k)
    fresh.set_option(cs.OPT_GRAPHS, graphs)
    ref_a = run(cs, torch, fresh, A, Ya, k, algo, prec)
    n_full = setup_launches(fresh)
    ref_b = run(cs, torch, fresh, A, Yb, k, algo, prec)

    plan = cs.Plan(m, n, B, k)
    plan.set_option(cs.OPT_GRAPHS, graphs)
    plan.set_A_generation(1)
    got = run(cs, torch, plan, A, Ya, k, algo, prec)
    assert setup_launches(plan) == n_full
    same(got, ref_a)
    skipped = None
    for rep in range(3):                       # eager, then (graphs on) capture and replay
        got = run(cs, torch, plan, A, Yb, k, algo, prec)
        same(got, ref_b)
        s = setup_launches(plan)
        assert s < n_full, "the preparation of A was not reused"
        skipped = n_full - s if skipped is None else skipped
        assert n_full - s == skipped
    # prep_A, plus A^T A where the fit or the Gram-form gathers use it
    assert skipped in (1, 2)

    # the oracle agrees with the reused solve
    if algo == "clomp":
        o = oracle.clomp(A64, Y64, k, steps=CL["steps"], lr=f32(CL["lr"]), beta1=f32(CL["beta1"]),
                         beta2=f32(CL["beta2"]), eps=f32(CL["eps"]))
    else:
        o = oracle.omp(A64, Y64, k)
    print(compare(run(cs, torch, plan, A, Ya, k, algo, prec), o))


def test_new_generation_reprepares(cs_gpu, torch):
    """A changed in place under the same pointer: a new generation prepares
    the new A; generation 0 prepares A in every solve."""
    cs = cs_gpu
    m, n, B, k = 64, 256, 200, 8
    p = workloads.random_problem(m, n, B, k, seed=143, snr_db=40.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    q = workloads.random_problem(m, n, B, k, seed=144, snr_db=40.0, values="pm")
    B32, Z32, B64, Z64 = f32_problem(q.A, q.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    Z = torch.from_numpy(Z32).cuda()

    plan = cs.Plan(m, n, B, k)
    plan.set_option(cs.OPT_GRAPHS, 0)
    plan.set_A_generation(7)
    run(cs, torch, plan, A, Y, k, "clomp", "bf16")
    n_full = setup_launches(plan)
    A.copy_(torch.from_numpy(B32).cuda())      # same buffer, new contents
    plan.set_A_generation(8)
    got = run(cs, torch, plan, A, Z, k, "clomp", "bf16")
    assert setup_launches(plan) == n_full
    fresh = cs.Plan(m, n, B, k)
    fresh.set_option(cs.OPT_GRAPHS, 0)
    same(got, run(cs, torch, fresh, A, Z, k, "clomp", "bf16"))
    o = oracle.clomp(B64, Z64, k, steps=CL["steps"], lr=f32(CL["lr"]), beta1=f32(CL["beta1"]),
                     beta2=f32(CL["beta2"]), eps=f32(CL["eps"]))
    print(compare(got, o))
    # generation 0 turns reuse off
    plan.profile(reset=True)
    plan.set_A_generation(0)
    for _ in range(2):
        run(cs, torch, plan, A, Z, k, "clomp", "bf16")
        assert setup_launches(plan) == n_full


def test_tv_prior_invalidates_gram(cs_gpu, torch):
    """The TV prior adds lambda (Delta D)^T (Delta D) to A^T A in place: the
    solve after it prepares A^T A again, and a TV solve never reuses it."""
    cs = cs_gpu
    m, n, B, k = 64, 200, 120, 8
    p = workloads.random_problem(m, n, B, k, seed=145, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    fresh = cs.Plan(m, n, B, k)
    fresh.set_option(cs.OPT_GRAPHS, 0)
    ref_plain = run(cs, torch, fresh, A, Y, k, "clomp", "bf16")
    n_plain = setup_launches(fresh)
    ref_tv = run(cs, torch, fresh, A, Y, k, "clomp", "bf16", tv_weight=0.5)
    n_tv = setup_launches(fresh)

    plan = cs.Plan(m, n, B, k)
    plan.set_option(cs.OPT_GRAPHS, 0)
    plan.set_A_generation(3)
    same(run(cs, torch, plan, A, Y, k, "clomp", "bf16"), ref_plain)
    assert setup_launches(plan) == n_plain
    for _ in range(2):
        same(run(cs, torch, plan, A, Y, k, "clomp", "bf16", tv_weight=0.5), ref_tv)
        assert setup_launches(plan) == n_tv
    same(run(cs, torch, plan, A, Y, k, "clomp", "bf16"), ref_plain)
    assert setup_launches(plan) == n_plain
    same(run(cs, torch, plan, A, Y, k, "clomp", "bf16"), ref_plain)
    assert setup_launches(plan) < n_plain


def test_host_buffer_keys_on_host_A(cs_gpu, torch):
    cs = cs_gpu
    m, n, B, k = 64, 256, 160, 8
    p = workloads.random_problem(m, n, B, k, seed=146, snr_db=40.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    ref = cs.clomp_solve_batched_host(A32, Y32, k, prec="bf16", plan=cs.Plan(m, n, B, k), **CL)
    plan = cs.Plan(m, n, B, k)
    plan.set_A_generation(1)
    plan.profile(reset=True)
    got1 = cs.clomp_solve_batched_host(A32, Y32, k, prec="bf16", plan=plan, **CL)
    n_full = setup_launches(plan)
    got2 = cs.clomp_solve_batched_host(A32, Y32, k, prec="bf16", plan=plan, **CL)
    assert setup_launches(plan) < n_full
    for g in (got1, got2):
        for q in ("support", "coef", "n_iter", "res_norm", "status"):
            assert np.array_equal(g[q], ref[q]), q
    # another host array with the same generation is a different A
    A2 = np.asfortranarray(A32.copy())
    cs.clomp_solve_batched_host(A2, Y32, k, prec="bf16", plan=plan, **CL)
    assert setup_launches(plan) == n_full
