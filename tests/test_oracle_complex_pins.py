"""Pins of the complex-Q oracle (oracle/complex_q.py) to facts fixed by the
paper and the mathematics, independent of the oracle's own formulas:
  - p = n with the unitary DFT: A *Q B is the t-product (circular convolution
    of tubes, computed by brute force) divided by sqrt(n), and real for real
    inputs (remark after Def. 3.2);
  - p < n with DFT rows: the product of real tensors can be complex (same
    remark), its tubes lie in range(Q) (Def. 3.1 is a projection, Sec. 3), and
    A *Q B + A *Q_perp B = A *M B with Q_perp the remaining DFT rows;
  - the truncated *Q-SVD over C meets the Eckart-Young identity of Thm. 4.2
    and the *Q-SVDII identity of Thm. 4.4;
  - a complex Q with zero imaginary part reproduces the real oracle (whose
    SVD is an independent one-sided Jacobi);
  - unitary invariance: multiplying Q's columns by unit phases leaves the
    approximation A_k unchanged (every singular value too)."""
import numpy as np
import pytest

import oracle
from oracle import complex_q as cq
from paper_2409_19402_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng(seed):
    return np.random.default_rng(seed)


def test_dft_q_has_unitary_columns():
    for n, p in ((8, 8), (12, 5), (7, 3)):
        Q = cq.dft_q(n, p)
        assert np.abs(Q.conj().T @ Q - np.eye(p)).max() <= 1e-13


def test_full_dft_gives_the_t_product():
    rng = _rng(1)
    n, n1, m, n2 = 8, 3, 4, 2
    A = rng.standard_normal((n, n1, m))
    B = rng.standard_normal((n, m, n2))
    C = cq.qprod_c(A, B, cq.dft_q(n, n))
    T = cq.tprod(A, B) / np.sqrt(n)
    np.testing.assert_allclose(C, T, atol=1e-12)
    assert np.abs(C.imag).max() <= 1e-12              # real for real inputs


def test_partial_dft_projection_split_and_complex_values():
    rng = _rng(2)
    n, n1, m, n2, p = 9, 3, 3, 2, 4
    A = rng.standard_normal((n, n1, m))
    B = rng.standard_normal((n, m, n2))
    F = cq.dft_q(n, n)
    Q, Qp = F[:, :p], F[:, p:]
    C = cq.qprod_c(A, B, Q)
    assert np.abs(C.imag).max() > 1e-3                  # complex, as the paper remarks
    P = np.eye(n) - Q @ Q.conj().T                      # tubes in range(Q)
    assert np.abs(cq.mode3_c(C, P)).max() <= 1e-12
    np.testing.assert_allclose(C + cq.qprod_c(A, B, Qp), cq.tprod(A, B) / np.sqrt(n), atol=1e-12)


def test_tsvdq_c_eckart_young_and_tsvdqII_identity():
    A = inputs.gaussian((12, 6, 5), seed=3).astype(np.float64)
    Q = cq.dft_q(12, 5)
    for k in (1, 3, 5):
        U, s, V, Ak, rep = cq.tsvdq_c(A, Q, k)
        assert rep.err2 == pytest.approx(rep.discarded2 + rep.proj_err2, rel=1e-12)
        assert rep.proj_err2 == pytest.approx(rep.normA2 - rep.normAh2, rel=1e-10)
        for t in range(Q.shape[1]):                      # orthonormal factors
            assert np.abs(U[t].conj().T @ U[t] - np.eye(k)).max() <= 1e-12
    for g in (0.5, 0.9, 0.99):
        rho, U, s, V, Ak, sig, rep = cq.tsvdqII_c(A, Q, g)
        assert rep.err2 == pytest.approx(rep.discarded2 + rep.proj_err2, rel=1e-12)
        kept = sum(float((st ** 2).sum()) for st in s)
        assert kept >= g * float((sig ** 2).sum()) * (1 - 1e-14)


def test_real_q_reduces_to_the_real_oracle():
    A = inputs.gaussian((10, 7, 6), seed=4).astype(np.float64)
    Qr = inputs.random_q(10, 4, seed=5).astype(np.float64)
    Uc, sc, Vc, Akc, repc = cq.tsvdq_c(A, Qr.astype(np.complex128), 3)
    Ur, sr, Vr, Akr, repr_ = oracle.tsvdq(A, Qr, 3)
    np.testing.assert_allclose(sc, sr, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Akc.real, Akr, atol=1e-12)
    assert np.abs(Akc.imag).max() <= 1e-12
    assert repc.err2 == pytest.approx(repr_.err2, rel=1e-10)


def test_column_phases_change_nothing():
    A = inputs.gaussian((8, 5, 4), seed=6).astype(np.float64)
    Q = cq.dft_q(8, 4)
    ph = np.exp(1j * np.array([0.3, -1.2, 2.0, 0.7]))
    _, s1, _, Ak1, _ = cq.tsvdq_c(A, Q, 2)
    _, s2, _, Ak2, _ = cq.tsvdq_c(A, Q * ph[None, :], 2)
    np.testing.assert_allclose(s1, s2, rtol=1e-12)
    np.testing.assert_allclose(Ak1, Ak2, atol=1e-12)
