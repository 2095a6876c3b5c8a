"""FP64 oracle of the column-wise 2D output path (test infrastructure, not
the product; the same import rules as the rest of ``oracle``).

* ``synthesize``: the image column x = D s from the solved sparse code s
  (Eq. 3 with the sparsifying basis D: the solver sees A = M D and returns s;
  the image is D s).
* ``psnr`` and ``ssim``: the two image-quality figures the paper reports for
  its reconstructions (Results).  The paper does not define them; this is
  the standard PSNR, 10 log10(L^2 / MSE), and the SSIM index of Wang, Bovik,
  Sheikh and Simoncelli (2004): an 11 x 11 Gaussian weighting window of
  standard deviation 1.5 normalised to unit sum, constants C1 = (0.01 L)^2
  and C2 = (0.03 L)^2, the index evaluated on every window that fits inside
  the image ("valid" placement) and averaged.  L is the dynamic range, by
  default max - min of the reference image.

Plain numpy in float64, written for reading, not speed.
"""
from __future__ import annotations

import math

import numpy as np

SSIM_SIZE = 11
SSIM_SIGMA = 1.5
SSIM_K1 = 0.01
SSIM_K2 = 0.03


def synthesize(D, support, coef, n_iter, n=None):
    """X[:, b] = sum over the first n_iter[b] support entries q of
    coef[b, q] * D[:, support[b, q]] (entries < 0 are skipped).  D None: the
    dense code itself (D = the n x n identity)."""
    D = np.eye(n) if D is None else np.asarray(D, dtype=np.float64)
    support = np.asarray(support)
    coef = np.asarray(coef, dtype=np.float64)
    B = support.shape[0]
    X = np.zeros((D.shape[0], B))
    for b in range(B):
        for q in range(int(n_iter[b])):
            j = int(support[b, q])
            if j >= 0:
                X[:, b] += coef[b, q] * D[:, j]
    return X


def gaussian_window(size=SSIM_SIZE, sigma=SSIM_SIGMA):
    c = (size - 1) / 2.0
    g = np.array([math.exp(-((i - c) ** 2) / (2.0 * sigma * sigma)) for i in range(size)])
    w = np.outer(g, g)
    return w / w.sum()


def _window_sums(img, w):
    """Weighted sums over every placement of w inside img (valid placement)."""
    H, W = img.shape
    r, c = w.shape
    out = np.zeros((H - r + 1, W - c + 1))
    for u in range(r):
        for v in range(c):
            out += w[u, v] * img[u:u + H - r + 1, v:v + W - c + 1]
    return out


def data_range(ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(ref.max() - ref.min())


def psnr(x, ref, L=None):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    L = data_range(ref) if L is None else float(L)
    mse = float(np.mean((x - ref) ** 2))
    return math.inf if mse == 0.0 else 10.0 * math.log10(L * L / mse)


def ssim(x, ref, L=None, window=None):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(ref, dtype=np.float64)
    L = data_range(y) if L is None else float(L)
    w = gaussian_window() if window is None else window
    C1 = (SSIM_K1 * L) ** 2
    C2 = (SSIM_K2 * L) ** 2
    mx = _window_sums(x, w)
    my = _window_sums(y, w)
    sxx = _window_sums(x * x, w) - mx * mx
    syy = _window_sums(y * y, w) - my * my
    sxy = _window_sums(x * y, w) - mx * my
    smap = ((2.0 * mx * my + C1) * (2.0 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(smap.mean())


def images_from_columns(X, W):
    """The consecutive H x W images held as the columns of X (H rows)."""
    X = np.asarray(X)
    return [X[:, i * W:(i + 1) * W] for i in range(X.shape[1] // W)]
