"""Seeded input generators: determinism, shapes and value ranges of the recipes."""
import numpy as np

from paper_2409_19402_gb300 import inputs


def test_tiny_shapes_and_determinism():
    A, B = inputs.tiny()
    assert A.shape == (16, 32, 24) and B.shape == (16, 24, 20)
    assert A.dtype == np.float32
    A2, _ = inputs.tiny()
    assert np.array_equal(A, A2)
    assert abs(float(A.std()) - 1.0) < 0.05


def test_video_recipe():
    V = inputs.video(l=24, m=32, n=20)
    assert V.shape == (20, 24, 32) and V.dtype == np.float32
    assert V.min() >= 0.0 and V.max() <= 1.0
    assert np.array_equal(V, inputs.video(l=24, m=32, n=20))


def test_hyperspectral_recipe():
    H = inputs.hyperspectral(l=16, m=16, n=30)
    assert H.shape == (30, 16, 16)
    assert np.array_equal(H, inputs.hyperspectral(l=16, m=16, n=30))


def test_batched_recipe():
    items = inputs.batched(count=3)
    for A, p in items:
        n, l, m = A.shape
        assert 32 <= l <= 256 and 32 <= m <= 256 and 64 <= n <= 512 and 8 <= p <= 64
        assert abs(float(np.sqrt((A.astype(np.float64) ** 2).mean())) - 1.0) < 0.01


def test_q_builders_orthonormal():
    for Q in (inputs.dct_q(16, 4), inputs.random_q(40, 7, seed=5),
              inputs.u3_q(inputs.video(l=12, m=16, n=30), 6)):
        G = Q.astype(np.float64).T @ Q.astype(np.float64)
        assert np.abs(G - np.eye(Q.shape[1])).max() < 1e-6
