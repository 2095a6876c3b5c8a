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
