"""GPU parity of the column-wise 2D output path -- x = D s from the sparse
codes, PSNR and SSIM -- against the FP64 oracle (oracle/image.py)."""
import numpy as np
import pytest

import oracle
from oracle import image as oi
import workloads
from parity import compare, f32, f32_problem, to_numpy

pytestmark = pytest.mark.gpu

CL = dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)

# SSIM tolerance: every window statistic is a float32 sum of 121 weighted
# terms (|error| <~ 121 * 2^-24 of the summed magnitudes, ~7e-6 relative),
# the centred second pass avoids cancellation, and the index's denominators
# are bounded below by C1 = (0.01 L)^2 and C2 = (0.03 L)^2; averaged over the
# windows the index moves by well under 1e-5.  PSNR: the squared errors are
# summed in float64, so only the float32 inputs and log10 matter.
SSIM_ATOL = 2e-5
PSNR_ATOL_DB = 1e-3


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def test_synthesize_matches_oracle(cs_gpu, torch):
    rng = np.random.default_rng(100)
    N, n, B, k = 256, 300, 37, 12
    D = rng.standard_normal((N, n)).astype(np.float32)
    support = np.stack([rng.choice(n, size=k, replace=False) for _ in range(B)]).astype(np.int32)
    coef = rng.standard_normal((B, k)).astype(np.float32)
    n_iter = rng.integers(0, k + 1, size=B).astype(np.int32)
    n_iter[0], n_iter[1] = k, 0
    support[2, 3] = -1                 # skipped
    support[3, 1] = n + 5              # outside [0, n): skipped
    n_iter[4] = k + 7                  # clamped to k
    Dt = torch.from_numpy(np.asfortranarray(D)).cuda()
    X = cs_gpu.synthesize(Dt, torch.from_numpy(support).cuda(), torch.from_numpy(coef).cuda(),
                          torch.from_numpy(n_iter).cuda())
    torch.cuda.synchronize()
    sup_o = support.copy()
    sup_o[sup_o >= n] = -1
    Xo = oi.synthesize(D.astype(np.float64), sup_o, coef.astype(np.float64), np.minimum(n_iter, k))
    np.testing.assert_allclose(X.cpu().numpy(), Xo, rtol=1e-5, atol=1e-5)
    assert np.all(X.cpu().numpy()[:, 1] == 0.0)


def _noisy_images(n_images, noise, seed):
    """The column-wise workload's images (H = 256, consecutive 256-column
    blocks) and a noisy copy."""
    ref = workloads.config_columnwise_2d(0.3, n_images=n_images).meta["X_img"]
    rng = np.random.default_rng(seed)
    x = ref + noise * ref.std() * rng.standard_normal(ref.shape)
    return np.asfortranarray(x, dtype=np.float32), np.asfortranarray(ref, dtype=np.float32)


@pytest.mark.parametrize("peak", [0.0, 1.5])
def test_image_quality_matches_oracle(cs_gpu, torch, peak):
    x, ref = _noisy_images(3, 0.2, seed=101)
    ps, ss = cs_gpu.image_quality(torch.from_numpy(x).cuda(), torch.from_numpy(ref).cuda(), 256, peak=peak)
    torch.cuda.synchronize()
    ps, ss = ps.cpu().numpy(), ss.cpu().numpy()
    for i, (xi, ri) in enumerate(zip(oi.images_from_columns(x, 256), oi.images_from_columns(ref, 256))):
        L = None if peak <= 0 else peak
        po = oi.psnr(xi.astype(np.float64), ri.astype(np.float64), L=L)
        so = oi.ssim(xi.astype(np.float64), ri.astype(np.float64), L=L)
        print(i, ps[i], po, ss[i], so)
        assert abs(ps[i] - po) < PSNR_ATOL_DB
        assert abs(ss[i] - so) < SSIM_ATOL


def test_image_quality_small_ragged_and_identical(cs_gpu, torch):
    rng = np.random.default_rng(102)
    H, W = 13, 17
    ref = rng.uniform(0.0, 255.0, size=(H, 2 * W)).astype(np.float32)
    x = np.clip(ref + rng.normal(0, 8.0, size=ref.shape), 0, 255).astype(np.float32)
    x[:, W:] = ref[:, W:]                      # the second image is exact
    ps, ss = cs_gpu.image_quality(torch.from_numpy(np.asfortranarray(x)).cuda(),
                                  torch.from_numpy(np.asfortranarray(ref)).cuda(), W, peak=255.0)
    torch.cuda.synchronize()
    ps, ss = ps.cpu().numpy(), ss.cpu().numpy()
    assert abs(ps[0] - oi.psnr(x[:, :W], ref[:, :W], L=255.0)) < PSNR_ATOL_DB
    assert abs(ss[0] - oi.ssim(x[:, :W].astype(np.float64), ref[:, :W].astype(np.float64), L=255.0)) < SSIM_ATOL
    assert ps[1] == np.inf and abs(ss[1] - 1.0) < 1e-6
    with pytest.raises(cs_gpu.CSError):
        cs_gpu.image_quality(torch.zeros((10, 20), device="cuda"), torch.zeros((10, 20), device="cuda"), 10)


def test_reconstruct_columnwise_end_to_end(cs_gpu, torch):
    """One 256 x 256 image at Sr = 0.3 (m = 77, k = 25): CLOMP solve of its
    256 columns, x = D s, PSNR / SSIM -- against the same pipeline on the
    FP64 oracle."""
    p = workloads.config_columnwise_2d(0.3, n_images=1)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    D32 = np.asfortranarray(p.meta["D"], dtype=np.float32)
    x_ref = p.meta["X_img"]
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    out = cs_gpu.reconstruct_columnwise(A, torch.from_numpy(D32).cuda(), Y, p.k, 256,
                                        ref=torch.from_numpy(np.asfortranarray(x_ref, dtype=np.float32)).cuda(),
                                        algo="clomp", prec="bf16", **CL)
    torch.cuda.synchronize()
    g = to_numpy(out["result"])
    p_ = {q: f32(v) for q, v in CL.items() if q != "steps"}
    o = oracle.clomp(A64, Y64, p.k, steps=CL["steps"], **p_)
    s = compare(g, o)
    Xo = oi.synthesize(D32.astype(np.float64), o["support"], o["coef"], o["n_iter"])
    Xg = out["X"].cpu().numpy()
    same = np.all(g["support"] == o["support"], axis=1)
    np.testing.assert_allclose(Xg[:, same], Xo[:, same], rtol=1e-4, atol=1e-5 * np.abs(Xo).max())
    po = oi.psnr(Xo, x_ref.astype(np.float32).astype(np.float64))
    so = oi.ssim(Xo, x_ref.astype(np.float32).astype(np.float64))
    pg, sg = float(out["psnr"].cpu()[0]), float(out["ssim"].cpu()[0])
    print(s, "psnr gpu/oracle", pg, po, "ssim gpu/oracle", sg, so)
    assert abs(pg - po) < 0.05 and abs(sg - so) < 1e-3


def test_dense_code_output(cs_gpu, torch):
    """Without a basis cs_synthesize writes the dense n x B code of a solve
    (the coefficients scattered to their atoms), equal to synthesising with
    the identity basis."""
    p = workloads.random_problem(64, 300, 40, 10, seed=103, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    r = cs_gpu.clomp_solve_batched(A, Y, 10, prec="bf16", **CL)
    X = cs_gpu.synthesize(None, r.support, r.coef, r.n_iter, n=300)
    Xi = cs_gpu.synthesize(torch.eye(300, device="cuda"), r.support, r.coef, r.n_iter)
    torch.cuda.synchronize()
    g = to_numpy(r)
    Xo = oi.synthesize(None, g["support"], g["coef"].astype(np.float64), g["n_iter"], n=300)
    assert np.array_equal(X.cpu().numpy(), Xo.astype(np.float32))
    assert np.array_equal(X.cpu().numpy(), Xi.cpu().numpy())
    assert np.count_nonzero(X.cpu().numpy()[:, 0]) == g["n_iter"][0]
