"""Seeded synthetic inputs for the projected t-SVD workloads.

This module only draws data and builds transformation matrices; it holds none
of the method's arithmetic (no mode-3 products, SVDs, truncation or rebuilds).
Both the CUDA path's tests/benchmark and the FP64 oracle consume exactly the
FP32 arrays returned here.

Tensor storage: an n1 x n2 x n3 tensor is a C-contiguous array of shape
(n3, n1, n2) -- frontal slice t (a video frame, a spectral band) is ``T[t]``.
All random draws use NumPy's PCG64 generator (``np.random.default_rng(seed)``),
in FP64, rounded to FP32 at the end.

Workloads (stand-ins for the paper's datasets, which are not available here):
  tiny           A 32x24x16, B 24x20x16 i.i.d. N(0,1)                    seed 0
  video          120x160x300 frames of 20 moving Gaussian blobs + noise   seed 1
                 (shape class of the traffic/shuttle videos, Sec. 5.2)
  hyperspectral  512x512x224 linear mixtures of 8 smooth spectra + noise  seed 2
                 (shape class of Indian Pines, Sec. 5.3)
  batched        64 Tucker-rank-10 tensors of uneven sizes + noise         seed 3
Transformation matrices (Sec. 5.1.1): DCT-II, random orthonormal, and U3 (the
leading left singular vectors of the mode-3 unfolding, Thm. 4.3); complex
ones (Sec. 3, Q in St_{n,p}(C)): the DFT rows and a random complex Q.
"""
from __future__ import annotations

import math

import numpy as np


def tiny(seed: int = 0):
    """A (32 x 24 x 16) and B (24 x 20 x 16), i.i.d. N(0,1); returns FP32 arrays
    of shapes (16, 32, 24) and (16, 24, 20)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((16, 32, 24))
    B = rng.standard_normal((16, 24, 20))
    return A.astype(np.float32), B.astype(np.float32)


def gaussian(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, scale^2) FP32 array of the given storage shape."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(shape)).astype(np.float32)


def video(seed: int = 1, l: int = 120, m: int = 160, n: int = 300, blobs: int = 20,
          noise_std: float = 0.01) -> np.ndarray:
    """Video-shaped tensor l x m x n (height x width x frames), values in [0, 1].

    20 Gaussian blobs, each with width sigma ~ U[4, 15] px, amplitude ~ U[0.3, 1],
    start position uniform over the frame and a constant velocity ~ U[-1, 1]
    px/frame per axis.  Frames are the sum of the blobs, divided by the global
    maximum, plus N(0, noise_std^2) noise (noise_std is the standard deviation),
    clipped to [0, 1].  Returned as FP32 of shape (n, l, m)."""
    rng = np.random.default_rng(seed)
    sig = rng.uniform(4.0, 15.0, blobs)
    amp = rng.uniform(0.3, 1.0, blobs)
    y0 = rng.uniform(0.0, l, blobs)
    x0 = rng.uniform(0.0, m, blobs)
    vy = rng.uniform(-1.0, 1.0, blobs)
    vx = rng.uniform(-1.0, 1.0, blobs)
    ii = np.arange(l, dtype=np.float64)[:, None]
    jj = np.arange(m, dtype=np.float64)[None, :]
    V = np.zeros((n, l, m))
    for t in range(n):
        frame = V[t]
        for b in range(blobs):
            cy, cx = y0[b] + vy[b] * t, x0[b] + vx[b] * t
            gy = np.exp(-((ii - cy) ** 2) / (2.0 * sig[b] ** 2))
            gx = np.exp(-((jj - cx) ** 2) / (2.0 * sig[b] ** 2))
            frame += amp[b] * (gy * gx)
    V /= V.max()
    V += noise_std * rng.standard_normal(V.shape)
    np.clip(V, 0.0, 1.0, out=V)
    return V.astype(np.float32)


def hyperspectral(seed: int = 2, l: int = 512, m: int = 512, n: int = 224,
                  endmembers: int = 8, noise_rel: float = 0.01) -> np.ndarray:
    """Hyperspectral-shaped tensor l x m x n (height x width x bands).

    8 endmember spectra, each a sum of 3 Gaussians over the band index (centre
    ~ U[0, n), width ~ U[5, 40], amplitude ~ U[0.2, 1]); each pixel mixes them
    with Dirichlet(0.5, ..., 0.5) abundances; Gaussian noise with standard
    deviation noise_rel * RMS(clean) is added.  Returned as FP32 (n, l, m)."""
    rng = np.random.default_rng(seed)
    bands = np.arange(n, dtype=np.float64)
    E = np.zeros((endmembers, n))
    for e in range(endmembers):
        c = rng.uniform(0.0, n, 3)
        w = rng.uniform(5.0, 40.0, 3)
        a = rng.uniform(0.2, 1.0, 3)
        for q in range(3):
            E[e] += a[q] * np.exp(-((bands - c[q]) ** 2) / (2.0 * w[q] ** 2))
    ab = rng.dirichlet(np.full(endmembers, 0.5), size=l * m)      # (l*m, endmembers)
    out = np.empty((n, l * m), dtype=np.float32)
    rms = None
    chunk = 1 << 15
    clean_sq = 0.0
    for s0 in range(0, l * m, chunk):                             # two passes keep memory low
        clean = ab[s0:s0 + chunk] @ E
        clean_sq += float((clean ** 2).sum())
    rms = math.sqrt(clean_sq / (l * m * n))
    for s0 in range(0, l * m, chunk):
        clean = ab[s0:s0 + chunk] @ E
        noisy = clean + noise_rel * rms * rng.standard_normal(clean.shape)
        out[:, s0:s0 + chunk] = noisy.T.astype(np.float32)
    return out.reshape(n, l, m)


def random_orthonormal(n: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """First p columns of the orthogonal factor of an n x n N(0,1) matrix (FP64),
    column signs fixed so that R has a non-negative diagonal."""
    G = rng.standard_normal((n, n))
    Qf, R = np.linalg.qr(G)
    Qf = Qf * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    return Qf[:, :p]


def batched(seed: int = 3, count: int = 64, noise_std: float = 1e-3, rank: int = 10):
    """64 independent tensors: l, m ~ U{32..256}, n ~ U{64..512}, p ~ U{8..64};
    A = G x_1 U1 x_2 U2 x_3 U3 with a 10x10x10 N(0,1) core and random orthonormal
    factors, scaled to unit RMS, plus N(0, noise_std^2).  Returns a list of
    (A (n, l, m) FP32, p)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        l = int(rng.integers(32, 257))
        m = int(rng.integers(32, 257))
        n = int(rng.integers(64, 513))
        p = int(rng.integers(8, 65))
        G = rng.standard_normal((rank, rank, rank))               # (a, b, c) core
        U1 = random_orthonormal(l, rank, rng)
        U2 = random_orthonormal(m, rank, rng)
        U3 = random_orthonormal(n, rank, rng)
        # storage (n, l, m): A[t, i, j] = sum_abc G[a,b,c] U1[i,a] U2[j,b] U3[t,c]
        A = np.einsum("abc,ia,jb,tc->tij", G, U1, U2, U3, optimize=True)
        A /= math.sqrt(float((A ** 2).mean()))
        A += noise_std * rng.standard_normal(A.shape)
        out.append((np.ascontiguousarray(A, dtype=np.float32), p))
    return out


# ------------------------------------------------------------ transformations
def dct_q(n: int, p: int) -> np.ndarray:
    """Q = C(1:p, :)^T for the orthonormal DCT-II matrix C of size n, i.e.
    Q[s, t] = c_t cos(pi (2s+1) t / (2n)), c_0 = sqrt(1/n), c_t = sqrt(2/n).
    FP32 (n, p)."""
    s = np.arange(n, dtype=np.float64)[:, None]
    t = np.arange(p, dtype=np.float64)[None, :]
    c = np.where(t == 0, math.sqrt(1.0 / n), math.sqrt(2.0 / n))
    return (c * np.cos(math.pi * (2.0 * s + 1.0) * t / (2.0 * n))).astype(np.float32)


def dft_qc(n: int, p: int) -> np.ndarray:
    """Complex Q = F(1:p, :)^H for the unitary DFT matrix F (F[t, s] =
    exp(-2 pi i t s / n) / sqrt(n)): Q[s, t] = exp(+2 pi i s t / n) / sqrt(n),
    complex64 (n, p) -- the t-product-like transformation (p = n: the t-product
    up to the factor 1/sqrt(n))."""
    s = np.arange(n, dtype=np.float64)[:, None]
    t = np.arange(p, dtype=np.float64)[None, :]
    ang = 2.0 * math.pi * ((s * t) % n) / n
    return ((np.cos(ang) + 1j * np.sin(ang)) / math.sqrt(n)).astype(np.complex64)


def random_qc(n: int, p: int, seed: int) -> np.ndarray:
    """Random complex Q with orthonormal columns: the first p columns of the
    unitary factor of an n x n complex Gaussian matrix (FP64 QR, column phases
    fixed so that R has a non-negative real diagonal), complex64 (n, p)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Qf, R = np.linalg.qr(G)
    d = np.diag(R)
    Qf = Qf * (np.conj(d) / np.abs(d))[None, :]
    return np.ascontiguousarray(Qf[:, :p]).astype(np.complex64)


def random_q(n: int, p: int, seed: int) -> np.ndarray:
    """Random orthonormal Q (first p columns of an orthogonal matrix), FP32 (n, p)."""
    return random_orthonormal(n, p, np.random.default_rng(seed)).astype(np.float32)


def u3_q(A: np.ndarray, p: int) -> np.ndarray:
    """Leading p left singular vectors of the mode-3 unfolding A_(3) (Thm. 4.3),
    from a LAPACK eigendecomposition of the FP64 Gram matrix A_(3) A_(3)^T;
    each column's largest-magnitude entry is made positive.  FP32 (n, p)."""
    n = A.shape[0]
    X = np.asarray(A, dtype=np.float64).reshape(n, -1)
    G = X @ X.T
    w, E = np.linalg.eigh(G)
    E = E[:, ::-1][:, :p]
    arg = np.abs(E).argmax(axis=0)
    E = E * np.sign(E[arg, np.arange(p)])[None, :]
    return np.ascontiguousarray(E).astype(np.float32)
