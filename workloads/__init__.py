"""Seeded synthetic inputs for the sparse-reconstruction hot path.

This module only draws random numbers and assembles the problem instances
y = A s + noise of Eq. (1)/(3); it contains none of the reconstruction
arithmetic (no correlation, selection, least squares or Adam).  Both the CPU
oracle tests and the GPU path take their inputs from here, so it is the one
piece of code they share.

Every generator returns float64 numpy arrays in column-major (Fortran) order:
``A`` is m x n (lda = m) and ``Y`` is m x B (ldy = m), matching the layout of
the C-ABI.  The workloads mirror the shapes the paper evaluates (synthetic 1D
signals with a Gaussian sensing matrix, Results "Evaluation with synthetic 1D
data"; column-wise processing of DCT-sparse images, Results "Evaluation with
synthetic 2D data"); none of the paper's datasets is used or needed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2501115920

# Configuration ids (1-based, in the order the workloads are listed).
CFG_SINGLE_FP64 = 1      # n=256, m=64, one noiseless 8-sparse signal
CFG_BATCHED = 2          # n=1024, m=256, 4096 signals, 32-sparse, 40 dB
CFG_COLUMNWISE_2D = 3    # 64 images 256x256 as 16384 columns, m = 26/77/128
CFG_LARGE_1D = 4         # n=65536, m=19661, 2000-sparse (not generated in full here)
CFG_UNEVEN = 5           # 2000 instances of uneven n, m, k


@dataclass
class Problem:
    """One batch of signals sharing a measurement matrix."""
    name: str
    A: np.ndarray                 # m x n, float64, Fortran order
    Y: np.ndarray                 # m x B, float64, Fortran order
    k: int                        # target sparsity (iterations)
    tol: float = 0.0              # stop when ||r||_2 <= tol
    max_iter: int = 200           # R of the paper
    X_true: np.ndarray | None = None   # n x B ground-truth coefficients (if known)
    cl: dict = field(default_factory=lambda: dict(steps=50, lr=1e-2, beta1=0.9,
                                                  beta2=0.999, eps=1e-8))
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def B(self) -> int:
        return self.Y.shape[1]


def rng_for(cfg_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + cfg_id + 1000 * salt)


def gaussian_matrix(rng, m, n, unit_columns=True, scale=None):
    """i.i.d. Gaussian sensing matrix; N(0, 1/m) unless `scale` is given."""
    s = (1.0 / math.sqrt(m)) if scale is None else scale
    A = rng.standard_normal((m, n)) * s
    if unit_columns:
        A /= np.linalg.norm(A, axis=0, keepdims=True)
    return np.asfortranarray(A)


def bernoulli_matrix(rng, m, n):
    """+-1/sqrt(m) Bernoulli sensing matrix."""
    A = (rng.integers(0, 2, size=(m, n)) * 2 - 1).astype(np.float64) / math.sqrt(m)
    return np.asfortranarray(A)


def sparse_coefficients(rng, n, B, k, values="gauss"):
    """n x B matrix with k non-zeros per column at uniformly random positions.

    values: "gauss" -> N(0,1); "pm" -> +-(1 + |N(0,1)|) with a random sign.
    """
    X = np.zeros((n, B))
    for b in range(B):
        idx = rng.choice(n, size=k, replace=False)
        if values == "gauss":
            v = rng.standard_normal(k)
        elif values == "pm":
            v = (1.0 + np.abs(rng.standard_normal(k))) * rng.choice([-1.0, 1.0], size=k)
        else:
            raise ValueError(values)
        X[idx, b] = v
    return np.asfortranarray(X)


def add_noise(rng, Y_clean, snr_db):
    """Per-signal white Gaussian noise at the given SNR:
    sigma^2 = ||A s||^2 / (m * 10^(SNR/10))."""
    if snr_db is None:
        return np.asfortranarray(Y_clean.copy())
    m = Y_clean.shape[0]
    p = np.sum(Y_clean * Y_clean, axis=0) / (m * 10.0 ** (snr_db / 10.0))
    noise = rng.standard_normal(Y_clean.shape) * np.sqrt(p)[None, :]
    return np.asfortranarray(Y_clean + noise)


def dct_synthesis(N):
    """Orthonormal DCT-II synthesis matrix D (x = D s); columns are the
    DCT-II basis vectors, D^T D = I."""
    x = np.arange(N)[:, None]
    u = np.arange(N)[None, :]
    D = np.cos(np.pi * (2 * x + 1) * u / (2.0 * N)) * math.sqrt(2.0 / N)
    D[:, 0] = 1.0 / math.sqrt(N)
    return D


def random_problem(m, n, B, k, seed, *, snr_db=None, values="gauss",
                   unit_columns=True, tol=0.0, max_iter=None, name="random"):
    """A generic seeded instance, used for ragged sizes and edge cases."""
    rng = np.random.default_rng(seed)
    A = gaussian_matrix(rng, m, n, unit_columns=unit_columns)
    X = sparse_coefficients(rng, n, B, min(k, n), values=values)
    Y = add_noise(rng, A @ X, snr_db)
    return Problem(name=name, A=A, Y=Y, k=k, tol=tol,
                   max_iter=(k if max_iter is None else max_iter), X_true=X)


def config_single_fp64() -> Problem:
    """n=256, m=64; A i.i.d. N(0,1/m) with unit columns; x 8-sparse with N(0,1)
    values at uniform positions; y = Ax noiseless; k=8, tol=1e-10."""
    rng = rng_for(CFG_SINGLE_FP64)
    A = gaussian_matrix(rng, 64, 256)
    X = sparse_coefficients(rng, 256, 1, 8, values="gauss")
    Y = np.asfortranarray(A @ X)
    return Problem(name="omp_single_n256_m64_k8", A=A, Y=Y, k=8, tol=1e-10,
                   max_iter=8, X_true=X)


def config_batched(B=4096) -> Problem:
    """n=1024, m=256, one shared Gaussian A with unit columns; B signals each
    32-sparse with values +-(1+|N(0,1)|); 40 dB SNR noise; CL fit with 50 Adam
    steps per iteration at lr 1e-2."""
    rng = rng_for(CFG_BATCHED)
    A = gaussian_matrix(rng, 256, 1024)
    X = sparse_coefficients(rng, 1024, B, 32, values="pm")
    Y = add_noise(rng, A @ X, 40.0)
    return Problem(name=f"batched_n1024_m256_k32_B{B}", A=A, Y=Y, k=32, tol=0.0,
                   max_iter=32, X_true=X,
                   cl=dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8))


def config_columnwise_2d(sr=0.3, n_images=64) -> Problem:
    """64 synthetic 256x256 images whose 2D-DCT coefficients are
    |N(0,1)| * (1+i+j)^-1.5 with random signs, processed as 256-long columns;
    A = Phi * D256 with Phi i.i.d. N(0,1/m); m = 26/77/128 for Sr = 0.1/0.3/0.5
    (256*Sr rounded to nearest); k = floor(m/3)."""
    N = 256
    m = int(math.floor(N * sr + 0.5))
    rng = rng_for(CFG_COLUMNWISE_2D, salt=int(round(sr * 10)))
    D = dct_synthesis(N)
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    decay = (1.0 + i + j) ** -1.5
    cols = []
    for _ in range(n_images):
        C = np.abs(rng.standard_normal((N, N))) * decay * rng.choice([-1.0, 1.0], size=(N, N))
        img = D @ C @ D.T          # inverse orthonormal 2D DCT
        cols.append(img)
    X_img = np.concatenate(cols, axis=1)          # 256 x (256 * n_images)
    Phi = rng.standard_normal((m, N)) / math.sqrt(m)
    A = np.asfortranarray(Phi @ D)
    Y = np.asfortranarray(Phi @ X_img)
    return Problem(name=f"colwise2d_sr{sr}_m{m}_B{Y.shape[1]}", A=A, Y=Y,
                   k=m // 3, tol=0.0, max_iter=m // 3,
                   meta=dict(sr=sr, images=n_images, X_img=X_img, D=D))


def config_large_1d(n=65536, m=19661, k=2000, block=4096) -> Problem:
    """One long 1-D signal: a 256 x 256 image flattened to n = 65536 and
    measured at rate 0.3 (m = 19661) by a dense Gaussian A with unit columns,
    held in float32 (about 5.2 GB) and drawn in column blocks; x is k-sparse
    with N(0,1) values at uniform positions; y = A x, noiseless.  The image is
    taken as k-sparse in the 2D DCT basis; since a Gaussian matrix times an
    orthonormal basis is again a Gaussian matrix, A stands for that product
    directly.  A is float32 here (the other generators return float64)."""
    rng = rng_for(CFG_LARGE_1D)
    A = np.empty((m, n), dtype=np.float32, order="F")
    for j0 in range(0, n, block):
        j1 = min(n, j0 + block)
        G = rng.standard_normal((j1 - j0, m), dtype=np.float32)
        G /= np.linalg.norm(G.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
        A[:, j0:j1] = G.T
    S = np.sort(rng.choice(n, size=k, replace=False))
    X = np.zeros((n, 1))
    X[S, 0] = rng.standard_normal(k)
    y = A[:, S].astype(np.float64) @ X[S, 0]
    return Problem(name=f"large1d_n{n}_m{m}_k{k}", A=A, Y=np.asfortranarray(y.reshape(-1, 1)), k=k, tol=0.0,
                   max_iter=k, X_true=X)


def config_uneven(n_instances=2000, n_classes=32):
    """Uneven batch: 32 size classes with n log-uniform in [512,16384]
    (rounded to 64), m/n uniform in [0.1,0.5] (rounded to 16), Gaussian A for
    even classes and +-1/sqrt(m) Bernoulli for odd ones; instances assigned
    uniformly to classes; k uniform in [0.01n, 0.1n]; 30 dB noise.
    Returns a list of (class A, list of (y, k)) without materialising more
    than one matrix per class."""
    rng = rng_for(CFG_UNEVEN)
    classes = []
    for c in range(n_classes):
        n = int(round(math.exp(rng.uniform(math.log(512), math.log(16384))) / 64.0)) * 64
        n = max(512, min(16384, n))
        m = max(16, int(round(n * rng.uniform(0.1, 0.5) / 16.0)) * 16)
        classes.append(dict(n=n, m=m, bernoulli=(c % 2 == 1)))
    assign = rng.integers(0, n_classes, size=n_instances)
    ks = [int(rng.integers(max(1, int(0.01 * classes[a]["n"])),
                           int(0.1 * classes[a]["n"]) + 1)) for a in assign]
    return classes, assign, ks


def uneven_class_data(classes, assign, ks, c, snr_db=30.0, dtype=np.float64):
    """Materialise size class c of config_uneven: its matrix A (m x n; Gaussian
    with unit columns for even classes, +-1/sqrt(m) Bernoulli for odd ones)
    and, for every instance assigned to it, (instance index, y, x_true) with
    x k-sparse N(0,1) at uniform positions and per-signal noise at snr_db.
    Each class has its own seed, so classes can be drawn one at a time."""
    cl = classes[c]
    rng = rng_for(CFG_UNEVEN, salt=c + 1)
    m, n = cl["m"], cl["n"]
    A = bernoulli_matrix(rng, m, n) if cl["bernoulli"] else gaussian_matrix(rng, m, n)
    items = []
    for i in np.nonzero(np.asarray(assign) == c)[0]:
        k = int(ks[i])
        x = sparse_coefficients(rng, n, 1, k, values="gauss")
        y = add_noise(rng, A @ x, snr_db)[:, 0]
        items.append((int(i), y, x[:, 0]))
    return np.asfortranarray(A, dtype=dtype), items


def named(name: str) -> Problem:
    if name == "c1":
        return config_single_fp64()
    if name == "c2":
        return config_batched()
    if name.startswith("c3"):
        sr = {"c3a": 0.1, "c3b": 0.3, "c3c": 0.5, "c3": 0.3}[name]
        return config_columnwise_2d(sr)
    raise KeyError(name)
