"""The FP8 (E4M3) tensor-core correlation: its product against a model of
the quantisation, the rounding bound the selection uses, and solver parity
with the FP64 oracle (supports identical, coefficients within 1e-5: the fit
stays float32), through the C ABI."""
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


def e4m3(v):
    """Round float64 values to E4M3 (3 mantissa bits, exponents down to -6,
    subnormal spacing 2^-9), nearest-even, saturating at 448."""
    a = np.abs(v)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    q = 2.0 ** (e - 3)
    r = np.minimum(np.round(a / q) * q, 448.0)
    return np.sign(v) * r


def quantise_columns(X32):
    """Per-column scale max|x| / 448 (float32) and the E4M3 codes of x / scale
    (the division in float32, as the kernels do)."""
    amax = np.abs(X32).max(axis=0).astype(np.float32)
    sc = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    codes = e4m3((X32 / sc[None, :]).astype(np.float32).astype(np.float64))
    return sc, codes


@pytest.mark.parametrize("m,n,B", [(256, 1024, 300), (77, 301, 133), (130, 520, 129)])
def test_fp8_product_matches_the_quantised_model(cs_gpu, torch, m, n, B):
    """C8 = sr sa (R8 . A8) against the same product in float64 from a model
    of the quantiser: the tensor core's fp32 accumulation stays within the
    m 2^-22 per-term bound the certificate assumes; and against the exact
    A^T R within the certificate's quantisation bound."""
    rng = np.random.default_rng(m + n)
    A32 = np.asfortranarray(workloads.gaussian_matrix(rng, m, n), dtype=np.float32)
    R32 = np.asfortranarray(rng.standard_normal((m, B)), dtype=np.float32)
    C = cs_gpu.correlate(torch.from_numpy(A32).cuda(), torch.from_numpy(R32).cuda(), prec="fp8")
    torch.cuda.synchronize()
    C = C.cpu().numpy().astype(np.float64)            # n x B
    sa, qa = quantise_columns(A32)
    sr, qr = quantise_columns(R32)
    Aq = qa * sa[None, :].astype(np.float64)
    Rq = qr * sr[None, :].astype(np.float64)
    model = Aq.T @ Rq
    absmag = np.abs(Aq).T @ np.abs(Rq)
    err = np.abs(C - model)
    bound = m * 2.0 ** -22 * absmag + 1e-30
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    # the certificate's bound against the exact product
    A64, R64 = A32.astype(np.float64), R32.astype(np.float64)
    exact = A64.T @ R64
    ea = np.linalg.norm(A64 - Aq, axis=0).max()
    er = np.linalg.norm(R64 - Rq, axis=0)
    cm = np.linalg.norm(A64, axis=0).max()
    rn = np.linalg.norm(R64, axis=0)
    delta = ea * (rn + er) + cm * er + m * (2.0 ** -22 + 2.0 ** -23) * (cm + ea) * (rn + er)
    assert np.all(np.abs(C - exact) <= delta[None, :])
    print(f"fp8 m={m}: max |C - model| / bound {np.max(err / bound):.3g}; "
          f"max |C - exact| / delta {np.max(np.abs(C - exact) / delta[None, :]):.3g}; "
          f"delta / ||a|| ||r|| {np.median(delta / (cm * rn)):.3g}")


def _solve(cs, torch, A32, Y32, k, algo, plan=None, **kw):
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    plan = plan or cs.Plan(A32.shape[0], A32.shape[1], Y32.shape[1], k)
    fn = cs.omp_solve_batched if algo == "omp" else cs.clomp_solve_batched
    r = fn(A, Y, k, prec="fp8", plan=plan, **kw)
    torch.cuda.synchronize()
    g = to_numpy(r)
    g["suspects"], g["errflags"] = plan.counters(reset=True)
    g["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    return g


def _oracle(A64, Y64, k, algo):
    if algo == "omp":
        return oracle.omp(A64, Y64, k)
    return oracle.clomp(A64, Y64, k, steps=CL["steps"], **{q: f32(v) for q, v in CL.items() if q != "steps"})


@pytest.mark.parametrize("algo", ["omp", "clomp"])
def test_fp8_batched_workload_every_signal(cs_gpu, torch, algo):
    """n = 1024, m = 256, 4096 signals, k = 32: every signal against the
    oracle; the suspects (atoms the FP8 candidates could not rule out,
    re-scored in float32) are counted."""
    p = workloads.config_batched()
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    kw = {} if algo == "omp" else dict(form="gram", **CL)
    g = _solve(cs_gpu, torch, A32, Y32, p.k, algo, **kw)
    assert g["errflags"] == 0 and g["launches"]["persist"] == 0
    s = compare({q: v for q, v in g.items() if q not in ("suspects", "errflags", "launches")},
                _oracle(A64, Y64, p.k, algo))
    print(algo, s, "picks with suspects:", g["suspects"], "of", p.B * p.k)


@pytest.mark.parametrize("algo", ["omp", "clomp"])
@pytest.mark.parametrize("case", ["ragged", "columnwise_sr0.3"])
def test_fp8_other_workloads(cs_gpu, torch, algo, case):
    if case == "ragged":
        p = workloads.random_problem(77, 301, 333, 12, seed=91, snr_db=30.0, values="pm")
        idx = None
    else:
        p = workloads.config_columnwise_2d(0.3, n_images=8)
        idx = np.arange(0, p.B, 8)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    kw = {} if algo == "omp" else dict(form="gram", **CL)
    g = _solve(cs_gpu, torch, A32, Y32, p.k, algo, **kw)
    assert g["errflags"] == 0
    o = _oracle(A64, Y64 if idx is None else Y64[:, idx], p.k, algo)
    s = compare({q: v for q, v in g.items() if q not in ("suspects", "errflags", "launches")}, o, idx=idx)
    print(case, algo, s, "picks with suspects:", g["suspects"])


def test_fp8_limits(cs_gpu, torch):
    """Beyond the tensor-core sizes the FP8 correlation is refused (it has no
    large-instance form); in an uneven batch such an instance is not solved."""
    A = torch.randn(300, 600, device="cuda")
    Y = torch.randn(300, 4, device="cuda")
    with pytest.raises(cs_gpu.CSError) as e:
        cs_gpu.omp_solve_batched(A, Y, 10, prec="fp8")
    assert e.value.code == -5
    p = workloads.random_problem(64, 256, 1, 8, seed=92, snr_db=30.0)
    As = torch.from_numpy(np.asfortranarray(p.A, dtype=np.float32)).cuda()
    ys = torch.from_numpy(np.float32(p.Y[:, 0])).cuda()
    outs = cs_gpu.omp_solve_varlen([(As, ys, 8), (A, Y[:, 0].contiguous(), 10)], prec="fp8",
                                   plan=cs_gpu.Plan(300, 600, 8, 16))
    torch.cuda.synchronize()
    assert int(outs[0].status[0]) == cs_gpu.SIG_REACHED_K
    assert int(outs[1].status[0]) == cs_gpu.SIG_UNSUPPORTED
