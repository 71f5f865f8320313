"""FP64 CPU oracle for projected products with a COMPLEX transformation
(Q in St_{n,p}(C), Sec. 3; the DFT case discussed after Def. 3.2).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s oracle legs use it;
the product path never imports it.

Plain NumPy complex128, written from the definitions:
  dft_q        Q = F(1:p, :)^H for the unitary DFT matrix F (F[t, s] =
               exp(-2 pi i t s / n) / sqrt(n)) -- the t-product-like choice
  mode3_c      Def. 2.2 over C:  Y(i,j,t) = sum_s M(t,s) X(i,j,s)
  facewise_c   Def. 2.3 over C
  qprod_c      Def. 3.1 over C:  A *Q B = ((A x_3 Q^H) ^ (B x_3 Q^H)) x_3 Q
  tprod        the t-product by its definition, circular convolution of tubes
               (used to pin qprod_c: with p = n and the unitary DFT,
               A *Q B = (A * B) / sqrt(n))
  tsvdq_c      Alg. 4.1 over C with the error terms of Thm. 4.2
  tsvdqII_c    Alg. 4.2 over C with the error terms of Thm. 4.4
The facewise matrix SVD (Alg. 4.1 step 3) uses LAPACK's complex SVD through
numpy.linalg.svd as a library step; singular values sorted descending.
The global energy order of Alg. 4.2 reuses the oracle's ``select_energy``
(singular values are real).  Storage as in the rest of the oracle: an
n1 x n2 x n3 tensor is an array of shape (n3, n1, n2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _c128(x) -> np.ndarray:
    return np.asarray(x).astype(np.complex128)


def dft_q(n: int, p: int) -> np.ndarray:
    """Q = F(1:p,:)^H, Q[s, t] = exp(+2 pi i s t / n) / sqrt(n), shape (n, p)."""
    s = np.arange(n)[:, None]
    t = np.arange(p)[None, :]
    return np.exp(2j * np.pi * s * t / n) / np.sqrt(n)


def mode3_c(X, M) -> np.ndarray:
    """Def. 2.2: Y(i,j,t) = sum_s M(t,s) X(i,j,s); X (n3, n1, n2), M (q, n3)."""
    X, M = _c128(X), _c128(M)
    n3 = X.shape[0]
    Y = np.zeros((M.shape[0],) + X.shape[1:], dtype=np.complex128)
    for t in range(M.shape[0]):
        for s in range(n3):
            Y[t] += M[t, s] * X[s]
    return Y


def facewise_c(A, B) -> np.ndarray:
    """Def. 2.3: C(:,:,t) = A(:,:,t) B(:,:,t)."""
    A, B = _c128(A), _c128(B)
    return np.stack([A[t] @ B[t] for t in range(A.shape[0])])


def qprod_c(A, B, Q) -> np.ndarray:
    """Def. 3.1: A *Q B = ((A x_3 Q^H) ^ (B x_3 Q^H)) x_3 Q."""
    Q = _c128(Q)
    QH = Q.conj().T
    return mode3_c(facewise_c(mode3_c(A, QH), mode3_c(B, QH)), Q)


def tprod(A, B) -> np.ndarray:
    """t-product: C(i,j,t) = sum_k sum_s A(i,k,s) B(k,j,(t - s) mod n3)."""
    A, B = _c128(A), _c128(B)
    n3 = A.shape[0]
    C = np.zeros((n3, A.shape[1], B.shape[2]), dtype=np.complex128)
    for t in range(n3):
        for s in range(n3):
            C[t] += A[s] @ B[(t - s) % n3]
    return C


@dataclass
class ReportC:
    normA2: float
    normAh2: float
    err2: float
    discarded2: float
    proj_err2: float
    K: int
    kappa: int


def _svd_slices(Ah):
    U, s, Vh = [], [], []
    for t in range(Ah.shape[0]):
        u, sv, vh = np.linalg.svd(Ah[t], full_matrices=False)
        U.append(u)
        s.append(sv)
        Vh.append(vh.conj().T)                      # V: columns are right singular vectors
    return U, np.array(s), Vh


def _terms(A, Q, Ah, Ahk):
    A = _c128(A)
    Q = _c128(Q)
    Ak = mode3_c(Ahk, Q)
    normA2 = float((np.abs(A) ** 2).sum())
    normAh2 = float((np.abs(Ah) ** 2).sum())
    err2 = float((np.abs(A - Ak) ** 2).sum())
    proj = A - mode3_c(mode3_c(A, Q.conj().T), Q)
    return Ak, normA2, normAh2, err2, float((np.abs(proj) ** 2).sum())


def tsvdq_c(A, Q, k: int):
    """Alg. 4.1 over C.  Returns (U list, s (p, k), V list, A_k complex, ReportC);
    U[t] is n1 x k, V[t] is n2 x k, A-hat_k(:,:,t) = U[t] diag(s[t]) V[t]^H."""
    Q = _c128(Q)
    Ah = mode3_c(A, Q.conj().T)
    U, s, V = _svd_slices(Ah)
    Uk = [u[:, :k] for u in U]
    Vk = [v[:, :k] for v in V]
    sk = s[:, :k]
    Ahk = np.stack([(Uk[t] * sk[t]) @ Vk[t].conj().T for t in range(Ah.shape[0])])
    Ak, nA, nAh, err2, perr = _terms(A, Q, Ah, Ahk)
    disc = float((s[:, k:] ** 2).sum())
    p = Ah.shape[0]
    return Uk, sk, Vk, Ak, ReportC(nA, nAh, err2, disc, perr, 0, k * p)


def tsvdqII_c(A, Q, gamma: float):
    """Alg. 4.2 over C.  Returns (rho, U list, s list, V list, A_k, sigma (p, b),
    ReportC) with slice t keeping rho[t] terms."""
    from . import select_energy
    Q = _c128(Q)
    Ah = mode3_c(A, Q.conj().T)
    U, s, V = _svd_slices(Ah)
    K, rho, kept2, total2 = select_energy(s, gamma)
    Uk = [U[t][:, :rho[t]] for t in range(len(U))]
    Vk = [V[t][:, :rho[t]] for t in range(len(V))]
    sk = [s[t, :rho[t]] for t in range(len(U))]
    Ahk = np.stack([(Uk[t] * sk[t]) @ Vk[t].conj().T for t in range(Ah.shape[0])])
    Ak, nA, nAh, err2, perr = _terms(A, Q, Ah, Ahk)
    # Thm. 4.4: the discarded energy is the sum of the squared singular values
    # every slice drops (its entries past rho[t]), summed directly
    disc = float(sum((s[t, rho[t]:] ** 2).sum() for t in range(s.shape[0])))
    return rho, Uk, sk, Vk, Ak, s, ReportC(nA, nAh, err2, disc, perr, int(K), int(np.sum(rho)))
