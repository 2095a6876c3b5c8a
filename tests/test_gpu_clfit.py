"""GPU checks of the CL fit forward / adjoint pair and its autograd wrapper:
gradient vs central differences of the loss, vs the FP64 oracle gradient,
and the fused Adam step vs the oracle's Adam."""
import numpy as np
import pytest

import oracle
import workloads
from parity import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _case(seed=31, m=96, n=300, B=64, t=12):
    rng = np.random.default_rng(seed)
    A = workloads.gaussian_matrix(rng, m, n).astype(np.float32)
    Y = rng.standard_normal((m, B)).astype(np.float32)
    S = np.stack([rng.choice(n, size=t, replace=False) for _ in range(B)]).astype(np.int32)
    s = rng.standard_normal((B, t)).astype(np.float32)
    return np.asfortranarray(A), np.asfortranarray(Y), S, s


def test_forward_adjoint_vs_oracle(cs_gpu, torch):
    A, Y, S, s = _case()
    At = torch.from_numpy(A).cuda()
    Yt = torch.from_numpy(Y).cuda()
    St = torch.from_numpy(S).cuda()
    R, loss = cs_gpu.clfit_forward(At, St, torch.from_numpy(s).cuda(), Yt)
    g = cs_gpu.clfit_adjoint(At, St, R)
    R, loss, g = R.cpu().numpy(), loss.cpu().numpy(), g.cpu().numpy()
    for b in range(Y.shape[1]):
        L, gr, r = oracle.clfit_loss_grad(A.astype(np.float64), S[b], s[b].astype(np.float64),
                                          Y[:, b].astype(np.float64))
        assert abs(loss[b] - L) <= 1e-5 * L
        assert np.linalg.norm(R[:, b] - r) <= 1e-5 * np.linalg.norm(r)
        assert np.linalg.norm(g[b] - gr) <= 1e-5 * np.linalg.norm(gr)


def test_autograd_matches_central_differences(cs_gpu, torch):
    from paper_2501_11592_gb300.clfit import CLFit
    A, Y, S, s = _case(seed=32, B=8, t=6)
    At = torch.from_numpy(A).cuda()
    Yt = torch.from_numpy(Y).cuda()
    St = torch.from_numpy(S).cuda()
    sv = torch.from_numpy(s).cuda().requires_grad_(True)
    w = torch.linspace(0.5, 1.5, 8, device="cuda")
    (CLFit.apply(sv, At, St, Yt) * w).sum().backward()
    g = sv.grad.cpu().numpy().astype(np.float64)
    # central differences of the (exactly quadratic) loss, evaluated by the
    # FP64 oracle so that only the GPU gradient carries float32 rounding
    h = 1e-3
    for b in range(8):
        for q in range(6):
            e = np.zeros(6)
            e[q] = h
            Lp = oracle.clfit_loss_grad(A.astype(np.float64), S[b], s[b] + e, Y[:, b].astype(np.float64))[0]
            Lm = oracle.clfit_loss_grad(A.astype(np.float64), S[b], s[b] - e, Y[:, b].astype(np.float64))[0]
            fd = float(w[b]) * (Lp - Lm) / (2 * h)
            assert abs(g[b, q] - fd) <= 1e-5 * max(1.0, abs(fd))


def test_fused_adam_step_vs_oracle(cs_gpu, torch):
    A, Y, S, s = _case(seed=33, B=16, t=8)
    At = torch.from_numpy(A).cuda()
    Yt = torch.from_numpy(Y).cuda()
    St = torch.from_numpy(S).cuda()
    sv = torch.zeros(16, 8, device="cuda")
    mo = torch.zeros(16, 8, device="cuda")
    ve = torch.zeros(16, 8, device="cuda")
    steps = 40
    for tau in range(1, steps + 1):
        R, _ = cs_gpu.clfit_forward(At, St, sv, Yt)
        cs_gpu.clfit_adam_step(At, St, sv, R, mo, ve, tau, lr=f32(1e-2))
    got = sv.cpu().numpy()
    for b in range(16):
        s_o, _, _, _ = oracle.clfit_adam(A.astype(np.float64), S[b], Y[:, b].astype(np.float64),
                                         np.zeros(8), np.zeros(8), np.zeros(8), 0, steps,
                                         lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
        assert np.linalg.norm(got[b] - s_o) <= 1e-5 * np.linalg.norm(s_o)


def test_gradient_at_large_signal_subconfig(cs_gpu, torch):
    """Gradient check at the large-signal workload's sub-configuration:
    n=4096, m=1024, support t=128, batch 1024.  The adjoint kernel's gradient
    matches the FP64 oracle gradient (sampled signals) and central
    differences of the kernel's own float32 loss."""
    rng = np.random.default_rng(34)
    m, n, t, B = 1024, 4096, 128, 1024
    A = np.asfortranarray(workloads.gaussian_matrix(rng, m, n).astype(np.float32))
    S = np.stack([rng.choice(n, size=t, replace=False) for _ in range(B)]).astype(np.int32)
    s = rng.standard_normal((B, t)).astype(np.float32)
    Y = np.asfortranarray(rng.standard_normal((m, B)).astype(np.float32) * 4.0)
    At = torch.from_numpy(A).cuda()
    Yt = torch.from_numpy(Y).cuda()
    St = torch.from_numpy(S).cuda()
    sv = torch.from_numpy(s).cuda()
    R, loss = cs_gpu.clfit_forward(At, St, sv, Yt)
    g = cs_gpu.clfit_adjoint(At, St, R).cpu().numpy()
    for b in range(0, B, 97):
        L, gr, _ = oracle.clfit_loss_grad(A.astype(np.float64), S[b], s[b].astype(np.float64),
                                          Y[:, b].astype(np.float64))
        assert np.linalg.norm(g[b] - gr) <= 1e-5 * np.linalg.norm(gr)
        assert abs(float(loss[b]) - L) <= 1e-5 * L
    # Central differences of the float32 loss along random unit directions.
    # The loss is quadratic, so the difference quotient has no truncation
    # error for any step h; its only error is the float32 rounding of the two
    # losses, at most (m + t) 2^-24 L each (a sum of m squares of residuals
    # formed with t FMAs), i.e. (m + t) 2^-24 (L+ + L-) / (2h) overall.
    h = 4.0
    dirs = rng.standard_normal((B, t)).astype(np.float32)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    d = torch.from_numpy(dirs).cuda()
    _, lp = cs_gpu.clfit_forward(At, St, sv + h * d, Yt)
    _, lm = cs_gpu.clfit_forward(At, St, sv - h * d, Yt)
    lp, lm = lp.double().cpu().numpy(), lm.double().cpu().numpy()
    fd = (lp - lm) / (2 * h)
    dd = np.sum(g.astype(np.float64) * dirs.astype(np.float64), axis=1)
    tol = 2 * (m + t) * 2.0 ** -24 * (lp + lm) / (2 * h) + 1e-5 * np.abs(dd)
    assert np.all(np.abs(fd - dd) <= tol), np.max(np.abs(fd - dd) / tol)
