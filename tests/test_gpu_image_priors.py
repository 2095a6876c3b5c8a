"""GPU parity of the image priors against the FP64 oracle: the total
variation of Eq. 6 and the local variation of Eq. 7 (image_width = W: the
batch is images of W consecutive columns whose Adam steps are coupled)."""
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


def gpu_solve(cs, torch, A32, Y32, k, W, prec="bf16", D32=None, graphs=1, **kw):
    m, n = A32.shape
    A = torch.from_numpy(np.asfortranarray(A32)).cuda()
    Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
    D = None if D32 is None else torch.from_numpy(np.asfortranarray(D32)).cuda()
    plan = cs.Plan(m, n, max(Y32.shape[1], 1), k)
    plan.set_option(cs.OPT_GRAPHS, graphs)
    cl = dict(CL)
    cl.update(kw)
    r = cs.clomp_solve_batched(A, Y, k, prec=prec, form="gram", plan=plan, D=D, image_width=W, **cl)
    torch.cuda.synchronize()
    assert plan.counters()[1] == 0
    out = to_numpy(r)
    out["launches"] = {ph: v[0] for ph, v in plan.profile(reset=True).items()}
    return out


def oracle_2d(A64, Y64, k, w, W, D64=None, **kw):
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in kw.items() if q in p})
    rest = {q: v for q, v in kw.items() if q in ("tol", "max_iter")}
    return oracle.clomp(A64, Y64, k, steps=kw.get("steps", CL["steps"]), tv_weight=f32(w), D=D64,
                        image_width=W, **rest, **p)


@pytest.mark.parametrize("W,images,prec", [(24, 4, "bf16"), (24, 4, "fp32"), (2, 7, "bf16"),
                                           (40, 2, "bf16"), (33, 2, "fp32"), (100, 1, "bf16")])
def test_image_prior_without_basis(cs_gpu, torch, W, images, prec):
    """x = s: the image is the coefficient array itself; W = 2 (two one-warp
    columns), widths that split over 2 and 4 CTAs of a cluster (33: one idle
    warp)."""
    k = 8
    p = workloads.random_problem(64, 200, W * images, k, seed=160 + W, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, prec=prec, tv_weight=0.5)
    assert g["launches"]["persist"] == 0 and g["launches"]["fit"] == k
    print(compare(g, oracle_2d(A64, Y64, k, 0.5, W)))


def test_image_prior_columnwise_dct_basis(cs_gpu, torch):
    """One 256 x 256 image of the column-wise workload (A = Phi D, D the
    orthonormal DCT): a cluster of 8 CTAs per image; the horizontal term,
    evaluated on the coefficients, against the oracle's pixel-space form."""
    p = workloads.config_columnwise_2d(0.3, n_images=1)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    D32 = np.asfortranarray(p.meta["D"], dtype=np.float32)
    w = 32.0
    g = gpu_solve(cs_gpu, torch, A32, Y32, p.k, 256, D32=D32, tv_weight=w)
    o = oracle_2d(A64, Y64, p.k, w, 256, D64=D32.astype(np.float64))
    print(compare(g, o))
    # the horizontal coupling moves the result away from the per-column prior
    g1 = gpu_solve(cs_gpu, torch, A32, Y32, p.k, 0, D32=D32, tv_weight=w)
    assert np.abs(g["coef"] - g1["coef"]).max() > 1e-4


def test_image_prior_stopped_columns_and_graph_replay(cs_gpu, torch):
    """Columns that reach the tolerance early stop and keep serving as
    neighbours; eager and replayed solves agree bit for bit."""
    k, W = 10, 16
    p = workloads.random_problem(48, 160, 3 * W, k, seed=170, snr_db=60.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    # a few columns with 3-sparse signals stop well before k
    rng = np.random.default_rng(171)
    for b in (1, 2, 17, 30, 47):
        s = np.zeros(160)
        s[rng.choice(160, 3, replace=False)] = rng.choice([-1.0, 1.0], 3) * (1 + rng.random(3))
        Y32[:, b] = (A32.astype(np.float64) @ s).astype(np.float32)
    Y64 = Y32.astype(np.float64)
    tol = 0.3                           # every residual of the oracle's run is >= 0.08 away
    g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, tv_weight=0.1, tol=tol, graphs=0, steps=200, lr=2e-2)
    o = oracle_2d(A64, Y64, k, 0.1, W, tol=tol, steps=200, lr=2e-2)
    assert (o["n_iter"] < k).sum() >= 3, o["n_iter"]
    print(compare(g, o))
    h = None
    for _ in range(3):                  # eager, capture, replay
        r = gpu_solve(cs_gpu, torch, A32, Y32, k, W, tv_weight=0.1, tol=tol, graphs=1, steps=200, lr=2e-2)
        if h is not None:
            for q in ("support", "coef", "n_iter", "status"):
                assert np.array_equal(r[q], h[q]), q
        h = r
    for q in ("support", "coef", "n_iter", "status"):
        assert np.array_equal(g[q], h[q]), q


def test_image_prior_wide_image(cs_gpu, torch):
    """W = 300 needs a cluster of 10 CTAs (beyond the portable 8): solved and
    checked against the oracle where the device allows such clusters, else
    refused with CS_ENOTSUP."""
    k, W = 6, 300
    p = workloads.random_problem(32, 96, W, k, seed=172, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    try:
        g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, tv_weight=0.4)
    except cs_gpu.CSError as e:
        assert e.code == cs_gpu.CS_ENOTSUP
        pytest.skip(f"clusters of 10 CTAs: {e}")
    print(compare(g, oracle_2d(A64, Y64, k, 0.4, W)))


def test_image_prior_limits(cs_gpu, torch):
    p = workloads.random_problem(40, 120, 30, 6, seed=173, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    cs = cs_gpu
    for bad in (dict(image_width=7),                            # 30 columns are not whole images
                dict(image_width=10, th=0.7, prec="fp32"),      # one atom per iteration only
                dict(image_width=1000)):                        # wider than 512
        kw = dict(prec="bf16", tv_weight=0.5)
        kw.update(bad)
        with pytest.raises(cs.CSError) as e:
            cs.clomp_solve_batched(A, Y, 6, **kw)
        assert e.value.code == cs.CS_ENOTSUP, bad
    with pytest.raises(cs.CSError) as e:
        cs.clomp_solve_batched(A, Y, 6, prec="bf16", tv_weight=0.5, image_width=-1)
    assert e.value.code == cs.CS_EINVAL
    # without a prior weight the width changes nothing
    a = to_numpy(cs.clomp_solve_batched(A, Y, 6, prec="bf16", image_width=10))
    b = to_numpy(cs.clomp_solve_batched(A, Y, 6, prec="bf16"))
    for q in ("support", "coef", "n_iter", "status"):
        assert np.array_equal(a[q], b[q]), q


# Local variation (Eq. 7) over the same images, alone and with the image TV

LV_EPS = 1e-4          # the binding's default smoothing of the window deviation


def oracle_img(A64, Y64, k, W, tv=0.0, lv=0.0, D64=None, lv_eps=LV_EPS, **kw):
    p = {q: f32(v) for q, v in CL.items() if q != "steps"}
    p.update({q: f32(v) for q, v in kw.items() if q in p})
    return oracle.clomp(A64, Y64, k, steps=kw.get("steps", CL["steps"]), tv_weight=f32(tv),
                        lv_weight=f32(lv), lv_eps=f32(lv_eps), D=D64, image_width=W, **p)


@pytest.mark.parametrize("W,images,tv,lv", [(24, 3, 0.0, 0.5), (24, 3, 0.5, 0.5), (40, 2, 0.0, 1.0),
                                            (100, 1, 0.3, 0.8), (3, 5, 0.0, 2.0)])
def test_local_variation_without_basis(cs_gpu, torch, W, images, tv, lv):
    """x = s (n = 200 pixels per column): windows across the CTA edges of 2-
    and 4-CTA clusters, with and without the image TV; W = 3 has one window
    column."""
    k = 8
    p = workloads.random_problem(64, 200, W * images, k, seed=180 + W, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, tv_weight=tv, lv_weight=lv)
    assert g["launches"]["persist"] == 0 and g["launches"]["fit"] == k
    print(compare(g, oracle_img(A64, Y64, k, W, tv=tv, lv=lv)))


@pytest.mark.parametrize("W,images,tv,lv", [(24, 3, 0.5, 0.5), (40, 2, 0.0, 1.0), (3, 5, 0.0, 2.0)])
def test_local_variation_plain_deviation_without_basis(cs_gpu, torch, W, images, tv, lv):
    """Eq. 7 as printed (eps = 0, the plain sample deviation) where it is
    well-conditioned: with x = s the pixels off the support are exact zeros,
    so a window is either exactly constant (no gradient on either side) or
    holds a support pixel and has a deviation of the order of the
    coefficients.  The test first checks that conditioning on the oracle (a
    1e-7 relative change of Y leaves its supports in place and moves its
    coefficients by < 1e-6), then compares."""
    k = 8
    p = workloads.random_problem(64, 200, W * images, k, seed=180 + W, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    o = oracle_img(A64, Y64, k, W, tv=tv, lv=lv, lv_eps=0.0)
    rng = np.random.default_rng(189)
    o2 = oracle_img(A64, Y64 * (1 + 1e-7 * rng.standard_normal(Y64.shape)), k, W, tv=tv, lv=lv, lv_eps=0.0)
    assert np.array_equal(o["support"], o2["support"])
    assert np.max(np.linalg.norm(o["coef"] - o2["coef"], axis=1) / np.linalg.norm(o["coef"], axis=1)) < 1e-6
    g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, tv_weight=tv, lv_weight=lv, lv_eps=0.0)
    print(compare(g, o))


def test_local_variation_columnwise_dct_strip(cs_gpu, torch):
    """A 256 x 64 strip of a column-wise image (A = Phi D, D the DCT): both
    image priors, pixels synthesised through D every step.  With the smoothed
    deviation the fit is well-conditioned: the test first checks that a 1e-7
    relative change of Y leaves the oracle's supports and (to 1e-6) its
    coefficients in place, then compares."""
    p = workloads.config_columnwise_2d(0.3, n_images=1)
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y[:, :64])
    D32 = np.asfortranarray(p.meta["D"], dtype=np.float32)
    D64 = D32.astype(np.float64)
    o = oracle_img(A64, Y64, p.k, 64, tv=32.0, lv=4.0, D64=D64)
    rng = np.random.default_rng(188)
    o2 = oracle_img(A64, Y64 * (1 + 1e-7 * rng.standard_normal(Y64.shape)), p.k, 64, tv=32.0, lv=4.0, D64=D64)
    assert np.array_equal(o["support"], o2["support"])
    assert np.max(np.linalg.norm(o["coef"] - o2["coef"], axis=1) / np.linalg.norm(o["coef"], axis=1)) < 1e-6
    g = gpu_solve(cs_gpu, torch, A32, Y32, p.k, 64, D32=D32, tv_weight=32.0, lv_weight=4.0)
    print(compare(g, o))
    g0 = gpu_solve(cs_gpu, torch, A32, Y32, p.k, 64, D32=D32, tv_weight=32.0)
    assert np.abs(g["coef"] - g0["coef"]).max() > 1e-3


def test_local_variation_general_basis_short_columns(cs_gpu, torch):
    """A general (non-orthonormal) basis of 5 rows: three window rows per
    column; the LV term needs no orthonormality."""
    rng = np.random.default_rng(185)
    k, W, n = 6, 12, 80
    p = workloads.random_problem(40, n, 2 * W, k, seed=186, snr_db=30.0, values="pm")
    A32, Y32, A64, Y64 = f32_problem(p.A, p.Y)
    D32 = np.asfortranarray(rng.standard_normal((5, n)) / np.sqrt(5), dtype=np.float32)
    g = gpu_solve(cs_gpu, torch, A32, Y32, k, W, D32=D32, lv_weight=1.5)
    print(compare(g, oracle_img(A64, Y64, k, W, lv=1.5, D64=D32.astype(np.float64))))


def test_local_variation_limits(cs_gpu, torch):
    p = workloads.random_problem(40, 300, 30, 6, seed=187, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    cs = cs_gpu
    with pytest.raises(cs.CSError) as e:          # no image width
        cs.clomp_solve_batched(A, Y, 6, prec="bf16", lv_weight=0.5)
    assert e.value.code == cs.CS_EINVAL
    with pytest.raises(cs.CSError) as e:          # 300 pixels per column (x = s)
        cs.clomp_solve_batched(A, Y, 6, prec="bf16", lv_weight=0.5, image_width=10)
    assert e.value.code == cs.CS_ENOTSUP
    for bad in (dict(lv_weight=float("nan")), dict(lv_weight=0.5, lv_eps=-1.0)):
        with pytest.raises(cs.CSError) as e:
            cs.clomp_solve_batched(A, Y, 6, prec="bf16", image_width=10, **bad)
        assert e.value.code == cs.CS_EINVAL, bad


def test_local_variation_plans_of_different_heights(cs_gpu, torch):
    """Two plans whose images need different shared memory, used in turn
    (the first plan's second solve reuses its launch check): the kernel's
    shared-memory limit set for one plan does not break the other."""
    cs = cs_gpu
    W, k = 40, 6
    probs, plans, first = {}, {}, {}
    for n in (200, 64):
        p = workloads.random_problem(48, n, 2 * W, k, seed=190 + n, snr_db=30.0, values="pm")
        probs[n] = f32_problem(p.A, p.Y)
        plans[n] = cs.Plan(48, n, 2 * W, k)
    for n in (200, 64, 200):
        A32, Y32, A64, Y64 = probs[n]
        A = torch.from_numpy(np.asfortranarray(A32)).cuda()
        Y = torch.from_numpy(np.asfortranarray(Y32)).cuda()
        r = to_numpy(cs.clomp_solve_batched(A, Y, k, prec="bf16", plan=plans[n], image_width=W, lv_weight=0.7,
                                            **CL))
        torch.cuda.synchronize()
        if n in first:
            for q in ("support", "coef", "n_iter", "status"):
                assert np.array_equal(r[q], first[n][q]), q
        else:
            print(compare(r, oracle_img(A64, Y64, k, W, lv=0.7)))
            first[n] = r


def test_image_priors_refused_by_the_uneven_batch_calls(cs_gpu, torch):
    """The uneven-batch calls regroup instances by size class, which would
    mix images: the image priors are refused there (CS_ENOTSUP)."""
    cs = cs_gpu
    p = workloads.random_problem(32, 96, 4, 4, seed=196, snr_db=30.0, values="pm")
    A32, Y32, _, _ = f32_problem(p.A, p.Y)
    A = torch.from_numpy(A32).cuda()
    inst = [(A, torch.from_numpy(np.ascontiguousarray(Y32[:, b])).cuda(), 4) for b in range(4)]
    for extra in (dict(tv_weight=0.5, image_width=2), dict(lv_weight=0.5, image_width=4)):
        params = cs._clomp_params(1, 0.0, None, "bf16", 0, 50, 1e-2, 0.9, 0.999, 1e-8, False, "gram", **extra)
        with pytest.raises(cs.CSError) as e:
            cs._varlen(cs.load().clomp_solve_varlen, inst, params, None, None)
        assert e.value.code == cs.CS_ENOTSUP, extra
