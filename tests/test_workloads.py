"""Seeded generators: shapes, determinism and the stated distributions."""
import numpy as np

import workloads


def test_single_signal_config():
    p = workloads.config_single_fp64()
    assert (p.m, p.n, p.B, p.k) == (64, 256, 1, 8)
    assert np.allclose(np.linalg.norm(p.A, axis=0), 1.0)
    assert np.count_nonzero(p.X_true) == 8
    assert np.allclose(p.Y, p.A @ p.X_true)
    q = workloads.config_single_fp64()
    assert np.array_equal(p.A, q.A) and np.array_equal(p.Y, q.Y)


def test_batched_config_noise_and_values():
    p = workloads.config_batched(B=256)
    assert (p.m, p.n, p.B, p.k) == (256, 1024, 256, 32)
    nz = p.X_true[p.X_true != 0]
    assert nz.size == 32 * 256 and np.all(np.abs(nz) >= 1.0)
    clean = p.A @ p.X_true
    snr = 10 * np.log10(np.sum(clean ** 2) / np.sum((p.Y - clean) ** 2))
    assert abs(snr - 40.0) < 0.5
    assert p.A.flags.f_contiguous and p.Y.flags.f_contiguous


def test_columnwise_2d_config():
    p = workloads.config_columnwise_2d(0.1, n_images=2)
    assert (p.m, p.n, p.B, p.k) == (26, 256, 512, 8)
    D = workloads.dct_synthesis(16)
    assert np.allclose(D.T @ D, np.eye(16))


def test_columnwise_2d_measurement_model():
    """A = Phi D and Y = Phi X: the column code s = D^T x reproduces y exactly,
    for each sampling rate's m (256 Sr rounded) and k = floor(m / 3)."""
    for sr, m in ((0.1, 26), (0.3, 77), (0.5, 128)):
        p = workloads.config_columnwise_2d(sr, n_images=1)
        assert (p.m, p.k, p.B) == (m, m // 3, 256)
        D = p.meta["D"]
        assert np.allclose(D.T @ D, np.eye(256), atol=1e-12)
        S = D.T @ p.meta["X_img"]
        assert np.allclose(p.A @ S, p.Y, atol=1e-10 * np.abs(p.Y).max())


def test_uneven_batch_covers_the_stated_ranges():
    """The uneven batch is drawn as stated -- n log-uniform in [512, 16384]
    (multiples of 64), m/n in [0.1, 0.5] (m a multiple of 16), k in
    [0.01 n, 0.1 n], Bernoulli A for odd classes -- and is not narrowed to
    what any kernel handles: the draws reach into the top of every range."""
    classes, assign, ks = workloads.config_uneven()
    assert len(classes) == 32 and len(assign) == 2000 and len(ks) == 2000
    n = np.array([c["n"] for c in classes])
    m = np.array([c["m"] for c in classes])
    assert np.all((n >= 512) & (n <= 16384) & (n % 64 == 0))
    assert np.all(m % 16 == 0)
    assert np.all(m / n >= 0.1 - 8.0 / n) and np.all(m / n <= 0.5 + 8.0 / n)
    assert n.max() >= 8192 and n.min() <= 1024
    assert (m / n).max() >= 0.4 and (m / n).min() <= 0.2
    assert [c["bernoulli"] for c in classes] == [c % 2 == 1 for c in range(32)]
    nk = n[np.asarray(assign)]
    k = np.asarray(ks)
    assert np.all(k >= np.maximum(1, (0.01 * nk).astype(int))) and np.all(k <= (0.1 * nk).astype(int))
    assert (k / nk).max() >= 0.09 and (k / nk).min() <= 0.02
    assert np.all(np.bincount(np.asarray(assign), minlength=32) > 0)
    c2, a2, k2 = workloads.config_uneven()
    assert c2 == classes and np.array_equal(a2, assign) and k2 == ks


def test_uneven_class_data_matrices_and_signals():
    classes, assign, ks = workloads.config_uneven()
    for c in (0, 1):                     # one Gaussian and one Bernoulli class
        A, items = workloads.uneven_class_data(classes, assign, ks, c)
        cl = classes[c]
        assert A.shape == (cl["m"], cl["n"]) and A.flags.f_contiguous
        if cl["bernoulli"]:
            assert np.allclose(np.abs(A), 1.0 / np.sqrt(cl["m"]))
        else:
            assert np.allclose(np.linalg.norm(A, axis=0), 1.0)
        assert [i for i, _, _ in items] == [int(i) for i in np.nonzero(np.asarray(assign) == c)[0]]
        clean = noise = 0.0
        for i, y, x in items:
            assert np.count_nonzero(x) == ks[i]
            clean += np.sum((A @ x) ** 2)
            noise += np.sum((y - A @ x) ** 2)
        assert abs(10 * np.log10(clean / noise) - 30.0) < 0.5
        A2, items2 = workloads.uneven_class_data(classes, assign, ks, c)
        assert np.array_equal(A, A2) and all(np.array_equal(u[1], v[1]) for u, v in zip(items, items2))


def test_large_1d_generator_on_a_reduced_size():
    """The long 1-D signal's recipe at a reduced size: float32 A drawn in
    column blocks with unit columns, a k-sparse N(0,1) x, y = A x noiseless."""
    p = workloads.config_large_1d(n=3000, m=900, k=90, block=700)
    assert p.A.dtype == np.float32 and p.A.shape == (900, 3000) and p.A.flags.f_contiguous
    assert np.allclose(np.linalg.norm(p.A.astype(np.float64), axis=0), 1.0, atol=1e-5)
    assert np.count_nonzero(p.X_true) == 90 and p.k == 90 and p.tol == 0.0
    assert np.allclose(p.Y[:, 0], p.A.astype(np.float64) @ p.X_true[:, 0], rtol=0, atol=1e-12)


def test_matrix_and_coefficient_helpers():
    rng = np.random.default_rng(3)
    B = workloads.bernoulli_matrix(rng, 50, 70)
    assert np.allclose(np.abs(B), 1.0 / np.sqrt(50))
    G = workloads.gaussian_matrix(rng, 40, 60, unit_columns=False)
    assert abs(np.var(G) * 40 - 1.0) < 0.1
    X = workloads.sparse_coefficients(rng, 100, 30, 7, values="pm")
    assert np.all(np.count_nonzero(X, axis=0) == 7)
    assert np.all(np.abs(X[X != 0]) >= 1.0)
    D = workloads.dct_synthesis(256)
    assert np.allclose(D.T @ D, np.eye(256), atol=1e-12)
