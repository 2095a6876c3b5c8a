"""Uneven batches (instances of different n, m, k with their own A) through
the varlen C-ABI entry points, against the FP64 oracle per instance."""
import numpy as np
import pytest

import oracle
import workloads
from parity import compare, f32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo,prec", [("omp", "fp32"), ("omp", "bf16"), ("clomp", "bf16")])
def test_uneven_batch_matches_oracle(cs_gpu, algo, prec):
    import torch
    classes, insts = workloads.uneven_batch(n_instances=160, seed=81)
    A32 = [np.asfortranarray(A, dtype=np.float32) for A in classes]
    At = [torch.from_numpy(A).cuda() for A in A32]
    items = [(At[c], torch.from_numpy(np.float32(y)).cuda(), k) for c, y, k, _ in insts]
    m_max = max(A.shape[0] for A in A32)
    n_max = max(A.shape[1] for A in A32)
    plan = cs_gpu.Plan(m_max, n_max, 64, 64)      # small batch_max: big groups run in chunks
    if algo == "omp":
        outs = cs_gpu.omp_solve_varlen(items, prec=prec, plan=plan)
    else:
        outs = cs_gpu.clomp_solve_varlen(items, prec=prec, plan=plan, steps=50, lr=1e-2)
    torch.cuda.synchronize()
    kw = dict(lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
    for (c, y, k, _), o in zip(insts, outs):
        A64 = A32[c].astype(np.float64)
        y64 = np.float32(y).astype(np.float64)
        ora = oracle.omp(A64, y64, k) if algo == "omp" else oracle.clomp(A64, y64, k, steps=50, **kw)
        g = {q: getattr(o, q).cpu().numpy() for q in ("support", "coef", "n_iter", "res_norm", "status")}
        compare(g, ora)
    _, errs = plan.counters(reset=True)
    assert errs == 0


def test_varlen_rejects_instances_beyond_the_plan(cs_gpu):
    import torch
    A = torch.randn(32, 100, device="cuda")
    y = torch.randn(32, device="cuda")
    plan = cs_gpu.Plan(16, 100, 8, 8)
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.omp_solve_varlen([(A, y, 4)], plan=plan)
    assert e.value.code == -1
