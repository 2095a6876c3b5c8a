"""The autotuner: every configuration it chooses between computes the same
bits, so a solve gives identical outputs with tuning on or off and with
either tensor-core tile width; it records one choice per size class and
reuses it."""
import numpy as np
import pytest

import workloads
from parity import f32_problem, to_numpy

pytestmark = pytest.mark.gpu

CL = dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _run(cs, torch, A32, Y32, k, algo, prec, tune=1, tile=0, persist=0):
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = cs.Plan(A32.shape[0], A32.shape[1], Y32.shape[1], k)
    plan.set_option(cs.OPT_AUTOTUNE, tune)
    plan.set_option(cs.OPT_TC_TILE, tile)
    plan.set_option(cs.OPT_PERSIST, persist)
    fn = cs.omp_solve_batched if algo == "omp" else cs.clomp_solve_batched
    kw = {} if algo == "omp" else dict(form="gram", **CL)
    outs = []
    for _ in range(3):              # eager (tunes), captured, replayed
        outs.append(to_numpy(fn(A, Y, k, prec=prec, plan=plan, **kw)))
        torch.cuda.synchronize()
    for o in outs[1:]:
        for q in o:
            assert np.array_equal(o[q], outs[0][q]), q
    return outs[0], plan.autotune_report()


def _same(a, b):
    for q in ("support", "coef", "n_iter", "res_norm", "status"):
        assert np.array_equal(a[q], b[q]), q


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_tile_width_gives_the_same_bits(cs_gpu, torch, algo, prec):
    p = workloads.random_problem(200, 1000, 700, 20, seed=95, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    t256, _ = _run(cs_gpu, torch, A32, Y32, p.k, algo, prec, tune=0, tile=256)
    t128, _ = _run(cs_gpu, torch, A32, Y32, p.k, algo, prec, tune=0, tile=128)
    tuned, rep = _run(cs_gpu, torch, A32, Y32, p.k, algo, prec, tune=1)
    _same(t256, t128)
    _same(t256, tuned)
    keys = [k for k in rep if k.startswith("tc-correlation tile")]
    assert len(keys) == 1 and rep[keys[0]] in (0, 1), rep


def test_large_path_configurations_give_the_same_bits(cs_gpu, torch):
    """More signals than one pass holds (so signals-per-pass choices differ)."""
    p = workloads.random_problem(600, 3000, 9, 90, seed=96, snr_db=30.0)
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    for prec in ("bf16", "fp32"):
        off, rep0 = _run(cs_gpu, torch, A32, Y32, p.k, "omp", prec, tune=0)
        on, rep1 = _run(cs_gpu, torch, A32, Y32, p.k, "omp", prec, tune=1)
        _same(off, on)
        assert not rep0
        keys = [k for k in rep1 if k.startswith("large correlation")]
        assert len(keys) == 1, rep1
        print(prec, rep1)
