"""FP64 CPU oracle for projected tensor-tensor products (arXiv 2409.19402).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2409_19402_gb300``) never imports it and
shares no code with it: the C source ``pp_oracle.c`` is compiled on its own
with gcc, and this module only marshals NumPy arrays into it.

Storage convention: an n1 x n2 x n3 tensor is a C-contiguous NumPy array of
shape (n3, n1, n2) -- frontal slice t is ``T[t]``, a row-major n1 x n2 matrix.
Matrices are C-contiguous (rows, cols).  Inputs of any float dtype are upcast
to float64 exactly (FP32 -> FP64 is exact).

Function -> passage it follows:
  mode3              Def. 2.2 (mode-3 product ``X x_3 M``)
  facewise           Def. 2.3 (facewise product)
  qprod              Def. 3.1 (projected product ``A *Q B``)
  mprod              Def. 2.4 (``*M`` product with M and M^{-1} given)
  svd                matrix SVD used in Alg. 4.1 step 3 (one-sided Jacobi)
  tsvdq              Alg. 4.1 + Thm. 4.2 error terms
  select_energy      Alg. 4.2 steps 4-7 (global order, K, rho)
  tsvdqII            Alg. 4.2 + Thm. 4.4 error terms
  sym_eig            symmetric eigensolver (HOSVD factors, U3)
  hosvd              truncated HOSVD of Sec. 4.2
  dct_q, householder_q, u3_q   transformation matrices of Sec. 5.1.1
  relative_error, compression_ratio   metrics RE and CR of Sec. 5.1.2
  qprod_grad         gradient of 1/2 |A *Q B - T|^2 w.r.t. A, B and Q (chain rule
                     through Def. 3.1; Q gradient also projected on the Stiefel
                     tangent space)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pp_oracle.c")
_LIB = os.path.join(_HERE, "_pp_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_pp_oracle_omp.so")   # same source, -fopenmp

OR_OK, OR_EINVAL, OR_ENOCONV, OR_ENOMEM = 0, 1, 5, 9


def build(force: bool = False) -> str:
    """Compile pp_oracle.c with gcc into oracle/_pp_oracle.so (no GPU needed), and
    the same source with -fopenmp into oracle/_pp_oracle_omp.so (the multi-core
    timing baseline; skipped where the compiler has no OpenMP)."""
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + f".tmp{os.getpid()}"
            r = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp,
                                _SRC, "-lm"], capture_output=True, text=True)
            if r.returncode != 0:
                if extra:          # no OpenMP: the single-thread library still serves
                    continue
                raise RuntimeError(f"gcc failed building the oracle:\n{r.stderr}")
            os.replace(tmp, lib)
    return _LIB


def has_openmp() -> bool:
    """The OpenMP build of the oracle exists (after build())."""
    build()
    return os.path.exists(_LIB_OMP)


_libs = {}


def _L(omp: bool = False):
    key = bool(omp)
    if key not in _libs:
        build()
        if key and not os.path.exists(_LIB_OMP):
            raise OracleError("the OpenMP build of the oracle is not available")
        lib = ctypes.CDLL(_LIB_OMP if key else _LIB)
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        ip32, ip64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        lib.or_mode3.argtypes = [dp, i64, i64, i64, dp, i64, dp]
        lib.or_facewise.argtypes = [dp, dp, i64, i64, i64, i64, dp]
        lib.or_qprod.argtypes = [dp, dp, dp, i64, i64, i64, i64, i64, dp]
        lib.or_mprod.argtypes = [dp, dp, dp, dp, i64, i64, i64, i64, dp]
        lib.or_svd_jacobi.argtypes = [dp, i64, i64, dp, dp, dp, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]
        lib.or_tsvdq.argtypes = [dp, dp, i64, i64, i64, i64, i64, ctypes.c_int,
                                 dp, dp, dp, dp, ctypes.c_void_p]
        lib.or_select_energy.argtypes = [dp, i64, i64, ctypes.c_double, ip64, ip32, dp, dp]
        lib.or_tsvdqII.argtypes = [dp, dp, i64, i64, i64, i64, ctypes.c_double, ctypes.c_int,
                                   ip32, ip64, dp, dp, dp, dp, dp, ctypes.c_void_p]
        lib.or_sym_eig_jacobi.argtypes = [dp, i64, dp, dp, ctypes.c_int]
        lib.or_mode_gram.argtypes = [dp, i64, i64, i64, ctypes.c_int, dp]
        lib.or_hosvd.argtypes = [dp, i64, i64, i64, i64, i64, dp, i64, dp, dp]
        lib.or_dct_q.argtypes = [i64, i64, dp]
        lib.or_qprod_grad.argtypes = [dp, dp, dp, dp, i64, i64, i64, i64, i64, dp, dp, dp, dp, dp]
        lib.or_qprod_grad.restype = ctypes.c_int
        lib.or_householder_q.argtypes = [dp, i64, i64, dp]
        for f in ("or_qprod", "or_mprod", "or_svd_jacobi", "or_tsvdq", "or_select_energy",
                  "or_tsvdqII", "or_sym_eig_jacobi", "or_hosvd", "or_householder_q"):
            getattr(lib, f).restype = ctypes.c_int
        _libs[key] = lib
    return _libs[key]


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != OR_OK:
        raise OracleError(f"{what} failed with oracle status {st}")


class _Report(ctypes.Structure):
    _fields_ = [("normA2", ctypes.c_double), ("normAh2", ctypes.c_double),
                ("err2", ctypes.c_double), ("discarded2", ctypes.c_double),
                ("proj_err2", ctypes.c_double), ("K", ctypes.c_int64),
                ("kappa", ctypes.c_int64), ("max_sweeps", ctypes.c_int),
                ("status", ctypes.c_int)]


@dataclass
class Report:
    normA2: float
    normAh2: float
    err2: float
    discarded2: float
    proj_err2: float
    K: int
    kappa: int
    max_sweeps: int

    @property
    def rel_err(self) -> float:
        """RE = |A - A_k|_F / |A|_F (Sec. 5.1.2)."""
        return float(np.sqrt(self.err2 / self.normA2)) if self.normA2 > 0 else 0.0


def _report(r: _Report) -> Report:
    return Report(r.normA2, r.normAh2, r.err2, r.discarded2, r.proj_err2, int(r.K),
                  int(r.kappa), int(r.max_sweeps))


# ---------------------------------------------------------------- products
def mode3(X, M) -> np.ndarray:
    """Def. 2.2: ``X x_3 M`` for X of shape (n3, n1, n2) and M of shape (q, n3)."""
    X, M = _f64(X), _f64(M)
    n3, n1, n2 = X.shape
    q = M.shape[0]
    assert M.shape == (q, n3)
    Y = np.empty((q, n1, n2))
    _L().or_mode3(_p(X), n1, n2, n3, _p(M), q, _p(Y))
    return Y


def facewise(A, B) -> np.ndarray:
    """Def. 2.3: facewise product of A (p, n1, m) and B (p, m, n2)."""
    A, B = _f64(A), _f64(B)
    p, n1, m = A.shape
    assert B.shape[0] == p and B.shape[1] == m
    n2 = B.shape[2]
    C = np.empty((p, n1, n2))
    _L().or_facewise(_p(A), _p(B), n1, m, n2, p, _p(C))
    return C


def qprod(A, B, Q) -> np.ndarray:
    """Def. 3.1: ``A *Q B`` with Q of shape (n3, p), orthonormal columns."""
    A, B, Q = _f64(A), _f64(B), _f64(Q)
    n3, n1, m = A.shape
    _, m2, n2 = B.shape
    assert m2 == m and B.shape[0] == n3
    p = Q.shape[1]
    assert Q.shape == (n3, p)
    C = np.empty((n3, n1, n2))
    _check(_L().or_qprod(_p(A), _p(B), _p(Q), n1, m, n2, n3, p, _p(C)), "qprod")
    return C


def mprod(A, B, M, Minv) -> np.ndarray:
    """Def. 2.4: ``A *M B`` with M and its inverse given explicitly."""
    A, B, M, Minv = _f64(A), _f64(B), _f64(M), _f64(Minv)
    n3, n1, m = A.shape
    n2 = B.shape[2]
    C = np.empty((n3, n1, n2))
    _check(_L().or_mprod(_p(A), _p(B), _p(M), _p(Minv), n1, m, n2, n3, _p(C)), "mprod")
    return C


# ---------------------------------------------------------------- SVDs
def svd(X, max_sweeps: int = 60):
    """One-sided Jacobi SVD of a matrix; returns (U, s, V, sweeps), X = U diag(s) V^T."""
    X = _f64(X)
    rows, cols = X.shape
    r = min(rows, cols)
    U, s, V = np.empty((rows, r)), np.empty(r), np.empty((cols, r))
    sw = ctypes.c_int(0)
    _check(_L().or_svd_jacobi(_p(X), rows, cols, _p(U), _p(s), _p(V), max_sweeps,
                              ctypes.byref(sw)), "svd")
    return U, s, V, sw.value


def tsvdq(A, Q, k: int, max_sweeps: int = 60):
    """Alg. 4.1.  Returns (Uh (p,l,k), s (p,k), Vh (p,m,k), Ak (n,l,m), Report)."""
    A, Q = _f64(A), _f64(Q)
    n, l, m = A.shape
    p = Q.shape[1]
    Uh, s, Vh = np.empty((p, l, k)), np.empty((p, k)), np.empty((p, m, k))
    Ak = np.empty((n, l, m))
    rep = _Report()
    _check(_L().or_tsvdq(_p(A), _p(Q), l, m, n, p, k, max_sweeps, _p(Uh), _p(s), _p(Vh),
                         _p(Ak), ctypes.byref(rep)), "tsvdq")
    return Uh, s, Vh, Ak, _report(rep)


def select_energy(sig, gamma: float):
    """Alg. 4.2 steps 4-7 on a (p, r) array of per-slice singular values.

    Returns (K, rho (p,) int32, kept energy, total energy)."""
    sig = _f64(sig)
    p, r = sig.shape
    K = ctypes.c_int64(0)
    rho = np.zeros(p, dtype=np.int32)
    kept, total = ctypes.c_double(0), ctypes.c_double(0)
    _check(_L().or_select_energy(_p(sig), p, r, float(gamma), ctypes.byref(K),
                                 rho.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.byref(kept), ctypes.byref(total)), "select_energy")
    return int(K.value), rho, kept.value, total.value


@dataclass
class TsvdqIIResult:
    rho: np.ndarray        # (p,) int32 per-slice ranks (the *Q-multirank kept)
    offs: np.ndarray       # (p+1,) int64 packing offsets
    Uh: list               # per slice, (l, rho_t)
    s: list                # per slice, (rho_t,)
    Vh: list               # per slice, (m, rho_t)
    Ak: np.ndarray         # (n, l, m)
    sig_all: np.ndarray    # (p, r) every singular value of every slice
    report: Report


def tsvdqII(A, Q, gamma: float, max_sweeps: int = 60, omp: bool = False) -> TsvdqIIResult:
    """Alg. 4.2 (*Q-SVDII) with energy parameter gamma in (0, 1].  omp=True runs
    the OpenMP build (slices and mode-3 output slices shared out over threads,
    OMP_NUM_THREADS; the same arithmetic per slice)."""
    A, Q = _f64(A), _f64(Q)
    n, l, m = A.shape
    p = Q.shape[1]
    r = min(l, m)
    rho = np.zeros(p, dtype=np.int32)
    offs = np.zeros(p + 1, dtype=np.int64)
    Uhp, sp, Vhp = np.empty(p * r * l), np.empty(p * r), np.empty(p * r * m)
    Ak, sig = np.empty((n, l, m)), np.empty((p, r))
    rep = _Report()
    _check(_L(omp).or_tsvdqII(_p(A), _p(Q), l, m, n, p, float(gamma), max_sweeps,
                           rho.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           _p(Uhp), _p(sp), _p(Vhp), _p(Ak), _p(sig), ctypes.byref(rep)),
           "tsvdqII")
    Uh, s, Vh = [], [], []
    for t in range(p):
        o, rt = int(offs[t]), int(rho[t])
        Uh.append(Uhp[l * o: l * o + l * rt].reshape(l, rt))
        s.append(sp[o: o + rt].copy())
        Vh.append(Vhp[m * o: m * o + m * rt].reshape(m, rt))
    return TsvdqIIResult(rho, offs, Uh, s, Vh, Ak, sig, _report(rep))


def sym_eig(G, max_sweeps: int = 100):
    """Cyclic Jacobi eigendecomposition of a symmetric matrix; (w desc, E columns)."""
    G = _f64(G)
    n = G.shape[0]
    w, E = np.empty(n), np.empty((n, n))
    _check(_L().or_sym_eig_jacobi(_p(G), n, _p(w), _p(E), max_sweeps), "sym_eig")
    return w, E


def mode_gram(A, d: int) -> np.ndarray:
    """Gram matrix A_(d) A_(d)^T of the mode-d unfolding (d in 1, 2, 3)."""
    A = _f64(A)
    n3, n1, n2 = A.shape
    nd = {1: n1, 2: n2, 3: n3}[d]
    G = np.empty((nd, nd))
    _L().or_mode_gram(_p(A), n1, n2, n3, d, _p(G))
    return G


def hosvd(A, k1: int, k2: int, U3):
    """Truncated HOSVD of Sec. 4.2 with mode-3 factor U3 (n3, k3); returns (A_k, err2)."""
    A, U3 = _f64(A), _f64(U3)
    n3, n1, n2 = A.shape
    k3 = U3.shape[1]
    Ak = np.empty((n3, n1, n2))
    err2 = ctypes.c_double(0)
    _check(_L().or_hosvd(_p(A), n1, n2, n3, k1, k2, _p(U3), k3, _p(Ak), ctypes.byref(err2)),
           "hosvd")
    return Ak, err2.value


# ---------------------------------------------------------------- Q builders
def dct_q(n: int, p: int) -> np.ndarray:
    """Q = C(1:p,:)^T for the orthonormal DCT-II matrix C of size n (Sec. 5.1.1)."""
    Q = np.empty((n, p))
    _L().or_dct_q(n, p, _p(Q))
    return Q


def householder_q(X, p: int) -> np.ndarray:
    """First p columns of the orthogonal factor of the square matrix X (Sec. 5.1.1)."""
    X = _f64(X)
    n = X.shape[0]
    Q = np.empty((n, p))
    _check(_L().or_householder_q(_p(X), n, p, _p(Q)), "householder_q")
    return Q


def u3_q(A, p: int):
    """Leading p left singular vectors of the mode-3 unfolding (Thm. 4.3), from the
    oracle's Jacobi eigensolver on A_(3) A_(3)^T; returns (Q, sigma_3 all n3)."""
    w, E = sym_eig(mode_gram(A, 3))
    return E[:, :p].copy(), np.sqrt(np.maximum(w, 0.0))


# ---------------------------------------------------------------- metrics
def relative_error(A, Atilde) -> float:
    """RE = |A - Atilde|_F / |A|_F (Sec. 5.1.2)."""
    A, At = _f64(A), _f64(Atilde)
    return float(np.sqrt(((A - At) ** 2).sum() / (A ** 2).sum()))


def storage_tsvdq(n1: int, n2: int, k: int, p: int) -> int:
    """st of the truncated *Q-SVD in the transform domain: n1 k p + k n2 p."""
    return n1 * k * p + k * n2 * p


def storage_tsvdqII(n1: int, n2: int, kappa: int) -> int:
    """st of the *Q-SVDII: kappa (n1 + n2)."""
    return kappa * (n1 + n2)


def storage_hosvd(n1: int, n2: int, n3: int, k1: int, k2: int, k3: int) -> int:
    """st of the truncated HOSVD: k1 k2 k3 + n1 k1 + n2 k2 + n3 k3."""
    return k1 * k2 * k3 + n1 * k1 + n2 * k2 + n3 * k3


def hosvd_matched_k2(n1: int, n2: int, n3: int, p: int, k: int, variant: int) -> int:
    """Sec. 5.3 storage matching, by exhaustive search: the largest k2 in
    1..n2 (variant 0, HOSVD multirank (n1, k2, p)) or 1..min(n1, n2) (variant 1,
    multirank (k2, k2, p)) whose HOSVD storage (U3 = Q counted) does not exceed
    the *Q-SVD storage with truncation k plus the n3 p of Q; 0 if none does."""
    budget = storage_tsvdq(n1, n2, k, p) + n3 * p
    best = 0
    top = n2 if variant == 0 else min(n1, n2)
    for k2 in range(1, top + 1):
        k1 = n1 if variant == 0 else k2
        if storage_hosvd(n1, n2, n3, k1, k2, p) <= budget:
            best = k2
    return best


def compression_ratio(n1: int, n2: int, n3: int, st_approx: int, st_q: int) -> float:
    """CR = st[A] / (st[A~] + st[Q]) with st[A] = n1 n2 n3 (Sec. 5.1.2)."""
    return float(n1 * n2 * n3) / float(st_approx + st_q)


def qprod_grad(A, B, Q, T):
    """Gradient of L = 1/2 |A *Q B - T|_F^2.  Returns (L, dA, dB, dQ_euclid, dQ_stiefel)."""
    A, B, Q, T = _f64(A), _f64(B), _f64(Q), _f64(T)
    n, n1, m = A.shape
    n2 = B.shape[2]
    p = Q.shape[1]
    dA, dB = np.empty_like(A), np.empty_like(B)
    dQE, dQ = np.empty((n, p)), np.empty((n, p))
    loss = ctypes.c_double(0)
    _check(_L().or_qprod_grad(_p(A), _p(B), _p(Q), _p(T), n1, m, n2, n, p, _p(dA), _p(dB),
                              _p(dQE), _p(dQ), ctypes.byref(loss)), "qprod_grad")
    return loss.value, dA, dB, dQE, dQ
