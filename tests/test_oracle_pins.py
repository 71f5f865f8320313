"""Pins for the FP64 oracle: values and identities fixed by the paper and by
mathematics, checked without reference to the CUDA path.

Each test names the passage it pins.  Together they are chosen so that a
plausible slip in the oracle (dropped term, wrong sign or index, transposed
operand, wrong tie rule) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests.conftest import GOLDEN

RNG = np.random.default_rng(12345)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _tube(v):
    return np.asarray(v, dtype=np.float64).reshape(-1, 1, 1)


# ------------------------------------------------------------ Appendix example
def _haar_setup():
    g = _golden("appendix_haar_example.json")
    s2 = math.sqrt(2.0)
    H4 = 0.5 * np.array([[{"sqrt2": s2, "-sqrt2": -s2}.get(x, x) if isinstance(x, str) else x
                          for x in row] for row in g["H4_times_2"]], dtype=np.float64)
    M = H4.T                      # M = H4^T (Appendix)
    p = g["p"]
    Q = M[:p, :].T                # M = [Q  Qperp]^H  ->  Q = M(1:p,:)^H
    Qp = M[p:, :].T
    return g, M, Q, Qp


def test_appendix_haar_products():
    """Appendix: a *M b, a *Q b, a *Qperp b printed tubes (exact)."""
    g, M, Q, Qp = _haar_setup()
    a, b = _tube(g["a"]), _tube(g["b"])
    np.testing.assert_allclose(oracle.mprod(a, b, M, M.T).ravel(), g["a_starM_b"], atol=1e-14)
    np.testing.assert_allclose(oracle.qprod(a, b, Q).ravel(), g["a_starQ_b"], atol=1e-14)
    np.testing.assert_allclose(oracle.qprod(a, b, Qp).ravel(), g["a_starQperp_b"], atol=1e-14)


def test_appendix_haar_projections():
    """Appendix eq. Q / Qperp: projected tubes a x3 QQ^T etc. (exact)."""
    g, M, Q, Qp = _haar_setup()
    a, b = _tube(g["a"]), _tube(g["b"])
    proj = lambda x, P: oracle.mode3(oracle.mode3(x, P.T), P).ravel()
    np.testing.assert_allclose(proj(a, Q), g["a_proj_Q"], atol=1e-14)
    np.testing.assert_allclose(proj(b, Q), g["b_proj_Q"], atol=1e-14)
    np.testing.assert_allclose(proj(a, Qp), g["a_proj_Qperp"], atol=1e-14)
    np.testing.assert_allclose(proj(b, Qp), g["b_proj_Qperp"], atol=1e-14)
    # eq. sum_proj_prod: *M = *Q + *Qperp
    np.testing.assert_allclose(oracle.qprod(a, b, Q) + oracle.qprod(a, b, Qp),
                               oracle.mprod(a, b, M, M.T), atol=1e-14)


# ------------------------------------------------------------ Example 4.1
def test_counterexample_4_1():
    """Example 4.1: squared errors 3 = 1 + 2 (Q = U3(:,1)) and 2 = 0 + 2 (Haar row)."""
    g = _golden("counterexample_4_1.json")
    A = np.asarray(g["slices"], dtype=np.float64)          # (n3, n1, n2)
    Qu = np.asarray(g["Q_U3"], dtype=np.float64)
    Qh = np.asarray(g["Q_haar_row1_over_sqrt2"], dtype=np.float64) / math.sqrt(2.0)
    _, _, _, _, r1 = oracle.tsvdq(A, Qu, g["k"])
    _, _, _, _, r2 = oracle.tsvdq(A, Qh, g["k"])
    assert r1.err2 == pytest.approx(g["err2_U3"], abs=1e-13)
    assert r1.discarded2 == pytest.approx(g["eckart_young_U3"], abs=1e-13)
    assert r1.proj_err2 == pytest.approx(g["projection_U3"], abs=1e-13)
    assert r2.err2 == pytest.approx(g["err2_haar"], abs=1e-13)
    assert r2.discarded2 == pytest.approx(g["eckart_young_haar"], abs=1e-13)
    assert r2.proj_err2 == pytest.approx(g["projection_haar"], abs=1e-13)
    Ah = oracle.mode3(A, Qh.T)[0]
    np.testing.assert_allclose(Ah, math.sqrt(2.0) * np.asarray(g["A_x3_H2row1_sqrt2_units"]),
                               atol=1e-15)


# ------------------------------------------------------------ library special cases
def test_mode3_matches_einsum():
    """Def. 2.2 against numpy.einsum: Y[t,i,j] = sum_s M[t,s] X[s,i,j]."""
    X = RNG.standard_normal((7, 5, 6))
    M = RNG.standard_normal((3, 7))
    np.testing.assert_allclose(oracle.mode3(X, M), np.einsum("ts,sij->tij", M, X), atol=1e-13)


def test_mode3_is_unfolding_product():
    """Def. 2.1/2.2: fold(M X_(3)) with X_(3)(:, J(i,j)) = vec(tube(i,j))."""
    n1, n2, n3, q = 4, 3, 5, 2
    X = RNG.standard_normal((n3, n1, n2))
    M = RNG.standard_normal((q, n3))
    X3 = np.zeros((n3, n1 * n2))
    for i in range(n1):
        for j in range(n2):
            X3[:, i + j * n1] = X[:, i, j]          # J(i,j) = i + (j-1) n1 (0-based)
    Y3 = M @ X3
    Y = np.zeros((q, n1, n2))
    for i in range(n1):
        for j in range(n2):
            Y[:, i, j] = Y3[:, i + j * n1]
    np.testing.assert_allclose(oracle.mode3(X, M), Y, atol=1e-13)


def test_facewise_matches_matmul():
    """Def. 2.3 against numpy.matmul per slice."""
    A = RNG.standard_normal((4, 5, 3))
    B = RNG.standard_normal((4, 3, 6))
    np.testing.assert_allclose(oracle.facewise(A, B), A @ B, atol=1e-13)


@pytest.mark.parametrize("shape", [(32, 24), (24, 32), (17, 17), (1, 9), (9, 1), (40, 7)])
def test_svd_matches_lapack(shape):
    """One-sided Jacobi SVD: singular values equal LAPACK's; X = U S V^T; U, V orthonormal."""
    X = RNG.standard_normal(shape)
    U, s, V, sweeps = oracle.svd(X)
    np.testing.assert_allclose(s, np.linalg.svd(X, compute_uv=False), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose((U * s) @ V.T, X, atol=1e-13)
    r = min(shape)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-13)
    assert np.all(np.diff(s) <= 0)


def test_svd_rank_deficient_and_zero():
    """Rank-deficient input: trailing singular values are 0; a zero matrix gives
    zero singular values and zero long-side vectors (length-4 rows here)."""
    X = np.outer(RNG.standard_normal(6), RNG.standard_normal(5))
    U, s, V, _ = oracle.svd(X)
    assert s[0] == pytest.approx(np.linalg.norm(X), rel=1e-13)
    assert np.all(s[1:] < 1e-13 * s[0])
    U0, s0, V0, sw = oracle.svd(np.zeros((3, 4)))
    assert np.all(s0 == 0) and np.all(V0 == 0) and sw <= 1


def test_sym_eig_matches_lapack():
    X = RNG.standard_normal((9, 9))
    G = X @ X.T
    w, E = oracle.sym_eig(G)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(G)[::-1], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(E @ np.diag(w) @ E.T, G, atol=1e-11)
    np.testing.assert_allclose(E.T @ E, np.eye(9), atol=1e-12)


def test_mode_gram_definitions():
    A = RNG.standard_normal((5, 4, 3))          # n3=5, n1=4, n2=3
    G1 = sum(A[t] @ A[t].T for t in range(5))
    G2 = sum(A[t].T @ A[t] for t in range(5))
    A3 = A.reshape(5, -1)
    np.testing.assert_allclose(oracle.mode_gram(A, 1), G1, atol=1e-12)
    np.testing.assert_allclose(oracle.mode_gram(A, 2), G2, atol=1e-12)
    np.testing.assert_allclose(oracle.mode_gram(A, 3), A3 @ A3.T, atol=1e-12)


# ------------------------------------------------------------ transformation matrices
def test_dct_q_closed_form_and_orthonormal():
    """Sec. 5.1.1 DCT: n = 2 gives the 2x2 Haar/DCT matrix; columns orthonormal."""
    Q2 = oracle.dct_q(2, 2)
    h = 1.0 / math.sqrt(2.0)
    np.testing.assert_allclose(Q2, [[h, h], [h, -h]], atol=1e-15)
    Q = oracle.dct_q(16, 4)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-14)
    # DCT-II of a cosine at frequency 3 concentrates in coefficient 3
    s = np.arange(16)
    x = np.cos(math.pi * (2 * s + 1) * 3 / 32)
    c = oracle.dct_q(16, 16).T @ x
    assert np.argmax(np.abs(c)) == 3 and np.sum(np.abs(c) > 1e-12) == 1


def test_householder_q():
    X = RNG.standard_normal((8, 8))
    Q = oracle.householder_q(X, 5)
    np.testing.assert_allclose(Q.T @ Q, np.eye(5), atol=1e-14)
    Qn, R = np.linalg.qr(X)
    Qn = Qn * np.sign(np.diag(R))[None, :]
    np.testing.assert_allclose(Q, Qn[:, :5], atol=1e-13)


# ------------------------------------------------------------ algebra (Sec. 3)
def _rand_q(n, p):
    return oracle.householder_q(RNG.standard_normal((n, n)), p)


def test_pequals_n_reduces_to_starM():
    """p = n, Q square orthogonal: A *Q B == A *M B with M = Q^T (Sec. 3.2),
    and both equal the brute-force tube-wise form eq. mprodEntrywise."""
    n = 6
    Q = _rand_q(n, n)
    M = Q.T
    A = RNG.standard_normal((n, 3, 4))
    B = RNG.standard_normal((n, 4, 2))
    C = oracle.qprod(A, B, Q)
    np.testing.assert_allclose(C, oracle.mprod(A, B, M, Q), atol=1e-12)
    # tube-wise: (A *M B)_{i,j,:} = sum_l A_{i,l,:} *M B_{l,j,:};  a *M b = M^{-1}((Ma).(Mb))
    Cb = np.zeros((n, 3, 2))
    for i in range(3):
        for j in range(2):
            for l in range(4):
                Cb[:, i, j] += Q @ ((M @ A[:, i, l]) * (M @ B[:, l, j]))
    np.testing.assert_allclose(C, Cb, atol=1e-12)


def test_tube_commutative_associative_distributive():
    """Thm. 3.1 and Thm. 3.2 on random tubes."""
    n, p = 7, 3
    Q = _rand_q(n, p)
    a, b, c = (RNG.standard_normal((n, 1, 1)) for _ in range(3))
    qp = lambda x, y: oracle.qprod(x, y, Q)
    np.testing.assert_allclose(qp(a, b), qp(b, a), atol=1e-13)
    np.testing.assert_allclose(qp(qp(a, b), c), qp(a, qp(b, c)), atol=1e-13)
    np.testing.assert_allclose(qp(a + b, c), qp(a, c) + qp(b, c), atol=1e-13)


def test_tensor_associativity():
    """Thm. 3.2 extended to compatibly sized tensors (proof's closing remark)."""
    n, p = 6, 4
    Q = _rand_q(n, p)
    A = RNG.standard_normal((n, 3, 4))
    B = RNG.standard_normal((n, 4, 5))
    C = RNG.standard_normal((n, 5, 2))
    qp = lambda x, y: oracle.qprod(x, y, Q)
    np.testing.assert_allclose(qp(qp(A, B), C), qp(A, qp(B, C)), atol=1e-12)


def _qtranspose(A, Q):
    """Def. 3.3 (real Q): transpose each transform-domain slice, then x_3 Q."""
    Ah = oracle.mode3(A, Q.T)
    return oracle.mode3(np.transpose(Ah, (0, 2, 1)).copy(), Q)


def test_transpose_of_product():
    """Thm. 3.3: (A *Q B)^H = B^H *Q A^H."""
    n, p = 6, 3
    Q = _rand_q(n, p)
    A = RNG.standard_normal((n, 3, 4))
    B = RNG.standard_normal((n, 4, 5))
    lhs = _qtranspose(oracle.qprod(A, B, Q), Q)
    rhs = oracle.qprod(_qtranspose(B, Q), _qtranspose(A, Q), Q)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_identity_and_its_nonuniqueness():
    """Def. 3.2 and eq. identityNull: I = I-hat x_3 Q acts as the identity on the
    projected space, and so does I + E x_3 (I - QQ^T)."""
    n, p, m = 6, 3, 4
    Q = _rand_q(n, p)
    Ihat = np.broadcast_to(np.eye(m), (p, m, m)).copy()
    I = oracle.mode3(Ihat, Q)
    A = RNG.standard_normal((n, 5, m))
    PA = oracle.mode3(oracle.mode3(A, Q.T), Q)                 # A x_3 QQ^T
    np.testing.assert_allclose(oracle.qprod(A, I, Q), PA, atol=1e-12)
    E = RNG.standard_normal((n, m, m))
    J = I + oracle.mode3(E, np.eye(n) - Q @ Q.T)
    np.testing.assert_allclose(oracle.qprod(A, J, Q), PA, atol=1e-12)
    # the second term vanishes in the transform domain
    np.testing.assert_allclose(oracle.mode3(J - I, Q.T), 0.0, atol=1e-12)


def test_split_identities_and_zero_slices():
    """eq. colSpaceDef, eq. sum_proj_prod and eq. backFrontalSlicesZero (with the
    second zero condition read as M(1:p,:), see the garble of that line)."""
    n, p = 7, 3
    Mfull = _rand_q(n, n).T                      # orthogonal M, rows are the transform
    Q, Qp = Mfull[:p].T, Mfull[p:].T
    A = RNG.standard_normal((n, 2, 3))
    B = RNG.standard_normal((n, 3, 4))
    PQ = Q @ Q.T
    lhs = oracle.qprod(A, B, Q)
    rhs = oracle.mprod(oracle.mode3(A, PQ), oracle.mode3(B, PQ), Mfull, Mfull.T)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    MB = oracle.mprod(A, B, Mfull, Mfull.T)
    np.testing.assert_allclose(lhs + oracle.qprod(A, B, Qp), MB, atol=1e-12)
    np.testing.assert_allclose(oracle.mode3(lhs, Mfull[p:]), 0.0, atol=1e-12)
    np.testing.assert_allclose(oracle.mode3(oracle.qprod(A, B, Qp), Mfull[:p]), 0.0, atol=1e-12)
    np.testing.assert_allclose(oracle.mode3(MB, Mfull[:p]), oracle.mode3(lhs, Q.T), atol=1e-12)


def test_w_equals_cq_scales_product():
    """Sec. 3.4: W = cQ with pseudoinverse reverse transform gives c (A *Q B)."""
    n, p, c = 5, 2, 3.0
    Q = _rand_q(n, p)
    W = c * Q
    A = RNG.standard_normal((n, 2, 3))
    B = RNG.standard_normal((n, 3, 2))
    Wpinv_T = np.linalg.pinv(W.T)               # (W^H)^dagger, n x p
    C = oracle.mode3(oracle.facewise(oracle.mode3(A, W.T), oracle.mode3(B, W.T)), Wpinv_T)
    np.testing.assert_allclose(C, c * oracle.qprod(A, B, Q), atol=1e-12)


# ------------------------------------------------------------ Sec. 4 theorems
def test_eckart_young_identity_and_optimality():
    """Thm. 4.2: |A - A_k|^2 = discarded sigma^2 + projection error (to 1e-12
    relative), and A_k beats random *Q-rank-k tensors X *Q Y^T."""
    n, l, m, p, k = 8, 6, 5, 4, 2
    A = RNG.standard_normal((n, l, m))
    Q = _rand_q(n, p)
    Uh, s, Vh, Ak, rep = oracle.tsvdq(A, Q, k)
    assert rep.err2 == pytest.approx(rep.discarded2 + rep.proj_err2, rel=1e-12)
    assert rep.err2 == pytest.approx(((A - Ak) ** 2).sum(), rel=1e-12)
    for _ in range(50):
        X = RNG.standard_normal((n, l, k))
        Y = RNG.standard_normal((n, m, k))
        B = oracle.qprod(X, _qtranspose(Y, Q), Q)
        assert ((A - B) ** 2).sum() >= rep.err2 * (1 - 1e-12)
    # perturbing the optimal factors never helps
    Ah_k = np.einsum("tir,tr,tjr->tij", Uh, s, Vh)
    for _ in range(20):
        Bp = oracle.mode3(Ah_k + 1e-3 * np.einsum("tir,tjr->tij", RNG.standard_normal(Uh.shape),
                                                  Vh), Q)
        assert ((A - Bp) ** 2).sum() >= rep.err2 * (1 - 1e-12)


def test_tsvdq_rebuild_from_factors():
    """Alg. 4.1: A_k = (U-hat_k S-hat_k V-hat_k^T) x_3 Q, factors orthonormal per slice."""
    n, l, m, p, k = 6, 5, 7, 3, 3
    A = RNG.standard_normal((n, l, m))
    Q = _rand_q(n, p)
    Uh, s, Vh, Ak, rep = oracle.tsvdq(A, Q, k)
    Ahk = np.einsum("tir,tr,tjr->tij", Uh, s, Vh)
    np.testing.assert_allclose(oracle.mode3(Ahk, Q), Ak, atol=1e-12)
    for t in range(p):
        np.testing.assert_allclose(Uh[t].T @ Uh[t], np.eye(k), atol=1e-12)
        np.testing.assert_allclose(Vh[t].T @ Vh[t], np.eye(k), atol=1e-12)
        sv = np.linalg.svd(oracle.mode3(A, Q.T)[t], compute_uv=False)
        np.testing.assert_allclose(s[t], sv[:k], rtol=1e-12)
        assert rep.discarded2 >= 0
    assert rep.discarded2 == pytest.approx(
        sum((np.linalg.svd(oracle.mode3(A, Q.T)[t], compute_uv=False)[k:] ** 2).sum()
            for t in range(p)), rel=1e-12)


def test_tsvdqII_identity_and_definition():
    """Thm. 4.4 error identity; Defs. 4.3/4.4 multirank and implicit rank."""
    n, l, m, p = 9, 6, 7, 4
    A = RNG.standard_normal((n, l, m))
    Q = _rand_q(n, p)
    res = oracle.tsvdqII(A, Q, 0.8)
    rep = res.report
    assert rep.err2 == pytest.approx(rep.discarded2 + rep.proj_err2, rel=1e-12)
    assert rep.kappa == res.rho.sum() == rep.K
    sig = res.sig_all
    kept = sum((sig[t, :res.rho[t]] ** 2).sum() for t in range(p))
    total = (sig ** 2).sum()
    assert kept >= 0.8 * total
    assert total == pytest.approx(rep.normAh2, rel=1e-12)   # energy denominator is |A-hat|^2
    # the K-1 largest values alone do not reach gamma
    flat = np.sort((sig ** 2).ravel())[::-1]
    assert flat[:rep.K - 1].sum() < 0.8 * total
    Ahk = np.zeros((p, l, m))
    for t in range(p):
        Ahk[t] = (res.Uh[t] * res.s[t]) @ res.Vh[t].T
    np.testing.assert_allclose(oracle.mode3(Ahk, Q), res.Ak, atol=1e-12)


def test_select_energy_hand_cases():
    """Alg. 4.2 steps 4-7 on hand-worked cases (golden)."""
    g = _golden("select_energy_cases.json")
    for c in g["cases"]:
        K, rho, kept, total = oracle.select_energy(np.asarray(c["sig"], float), c["gamma"])
        assert K == c["K"], c
        assert list(rho) == c["rho"], c


def test_select_gamma_one_keeps_all_nonzero():
    sig = np.abs(RNG.standard_normal((5, 6)))
    sig = -np.sort(-sig, axis=1)
    sig[:, 4:] = 0.0
    K, rho, _, _ = oracle.select_energy(sig, 1.0)
    assert K <= 20 and np.all(rho <= 4)


def test_tsvdqII_no_worse_than_tsvdq():
    """Thm. 4.5: gamma = |A_k x3 Q^T|^2 / |A x3 Q^T|^2 gives an error <= the *Q-SVD's."""
    n, l, m, p, k = 10, 7, 6, 5, 2
    A = RNG.standard_normal((n, l, m))
    Q = _rand_q(n, p)
    Uh, s, Vh, Ak, rep = oracle.tsvdq(A, Q, k)
    gamma = (s ** 2).sum() / rep.normAh2
    res = oracle.tsvdqII(A, Q, gamma * (1 - 1e-12))
    assert res.report.err2 <= rep.err2 * (1 + 1e-12)
    assert res.report.kappa <= k * p


def test_corollary_4_1_and_thm_4_3_u3():
    """Cor. 4.1 (Q = U3: projection error = sum_{j>p} sigma_j(A_(3))^2 and
    |A-hat_i|_F = sigma_i(A_(3))) and Thm. 4.3 (U3 minimises projection error)."""
    n, l, m, p = 8, 5, 6, 3
    A = RNG.standard_normal((n, l, m))
    Q, _ = oracle.u3_q(A, p)
    sv3 = np.linalg.svd(A.reshape(n, -1), compute_uv=False)      # LAPACK, independent
    _, _, _, _, rep = oracle.tsvdq(A, Q, 2)
    assert rep.proj_err2 == pytest.approx((sv3[p:] ** 2).sum(), rel=1e-10)
    Ah = oracle.mode3(A, Q.T)
    np.testing.assert_allclose(np.sqrt((Ah ** 2).sum(axis=(1, 2))), sv3[:p], rtol=1e-10)
    for _ in range(100):
        Qr = _rand_q(n, p)
        P = np.eye(n) - Qr @ Qr.T
        assert (oracle.mode3(A, P) ** 2).sum() >= rep.proj_err2 * (1 - 1e-12)


def test_starQ_rank_le_starM_rank():
    """Thm. 4.1 on a tensor whose *M transform slices have ranks 1..n."""
    n, l, m, p = 5, 6, 6, 2
    M = _rand_q(n, n).T
    Ahat = np.zeros((n, l, m))
    for t in range(n):
        Ahat[t] = RNG.standard_normal((l, t + 1)) @ RNG.standard_normal((t + 1, m))
    A = oracle.mode3(Ahat, M.T)                                  # A x_3 M = Ahat
    Q = M[:p].T
    rk = lambda X: int((oracle.svd(X)[1] > 1e-10 * np.linalg.norm(X)).sum())
    rq = max(rk(s) for s in oracle.mode3(A, Q.T))
    rm = max(rk(s) for s in oracle.mode3(A, M))
    assert rq == p and rm == n and rq <= rm


def test_hosvd_bound_thm_4_6():
    """Thm. 4.6: with Q = U3(:,1:p), k = min(k1,k2): *Q-SVD error <= HOSVD(k1,k2,p) error."""
    n, l, m, p = 9, 7, 6, 4
    A = RNG.standard_normal((n, l, m)) + 3 * np.einsum(
        "t,i,j->tij", RNG.standard_normal(n), RNG.standard_normal(l), RNG.standard_normal(m))
    Q, _ = oracle.u3_q(A, p)
    for k1, k2 in [(3, 2), (2, 5), (4, 4), (7, 6)]:
        _, hos_err2 = oracle.hosvd(A, k1, k2, Q)
        _, _, _, _, rep = oracle.tsvdq(A, Q, min(k1, k2))
        assert rep.err2 <= hos_err2 * (1 + 1e-12)


def test_hosvd_full_rank_is_projection():
    """HOSVD with k1 = n1, k2 = n2 reduces to the mode-3 projection A x_3 QQ^T."""
    n, l, m, p = 6, 4, 5, 3
    A = RNG.standard_normal((n, l, m))
    Q = _rand_q(n, p)
    Ak, err2 = oracle.hosvd(A, l, m, Q)
    np.testing.assert_allclose(Ak, oracle.mode3(oracle.mode3(A, Q.T), Q), atol=1e-12)


def _orth(n, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def test_hosvd_truncation_exact_on_a_diagonal_tucker_core():
    """Sec. 4.2 truncated HOSVD on A = G x1 U1 x2 U2 x3 U3 with a superdiagonal
    core G(r,r,r) = g_r, g strictly decreasing, and random orthogonal U_i (none
    symmetric): the mode-1 and mode-2 Grams are U_i diag(g^2) U_i^T, so the
    leading k_i eigenvectors are the first k_i columns of U_i, and with Q = U3
    (first p columns) the HOSVD(k1, k2, p) approximation is exactly
    sum_{r < min(k1, k2, p)} g_r u1_r o u2_r o u3_r with squared error
    sum_{r >= min(k1, k2, p)} g_r^2.  Trailing eigenvectors, or eigenvector
    matrices read by rows instead of columns, give other tensors and errors."""
    n1, n2, n3, p = 7, 6, 8, 4
    g = np.array([10.0, 7.0, 5.0, 3.0, 2.0, 1.5])
    U1, U2, U3 = _orth(n1, 31), _orth(n2, 32), _orth(n3, 33)
    R = len(g)
    A = np.einsum("r,ir,jr,tr->tij", g, U1[:, :R], U2[:, :R], U3[:, :R])
    Q = U3[:, :p]
    for k1, k2 in [(1, 6), (2, 3), (3, 2), (4, 4), (5, 6), (7, 6)]:
        kk = min(k1, k2, p)
        ref = np.einsum("r,ir,jr,tr->tij", g[:kk], U1[:, :kk], U2[:, :kk], U3[:, :kk])
        Ak, err2 = oracle.hosvd(A, k1, k2, Q)
        np.testing.assert_allclose(Ak, ref, atol=1e-11)
        assert err2 == pytest.approx(float(np.sum(g[kk:] ** 2)), rel=1e-10, abs=1e-10)


def test_hosvd_matches_svd_of_the_unfoldings():
    """Sec. 4.2 truncated HOSVD against the same construction from LAPACK's SVD
    of the mode-1 and mode-2 unfoldings (leading k_i left singular vectors):
    A_k = A x1 U1 U1^T x2 U2 U2^T x3 Q Q^T, |A - A_k|^2 = |A|^2 - |core|^2 with
    core = A x1 U1^T x2 U2^T x3 Q^T (orthogonal projections).  Random data has
    distinct singular values, so the truncated subspaces and A_k are unique."""
    n1, n2, n3, p = 9, 7, 10, 5
    A = RNG.standard_normal((n3, n1, n2))
    Q = _orth(n3, 41)[:, :p]
    A1 = A.transpose(1, 0, 2).reshape(n1, -1)       # mode-1 unfolding (i, (t, j))
    A2 = A.transpose(2, 0, 1).reshape(n2, -1)       # mode-2 unfolding (j, (t, i))
    W1 = np.linalg.svd(A1)[0]
    W2 = np.linalg.svd(A2)[0]
    for k1, k2 in [(3, 2), (2, 5), (6, 6), (9, 7)]:
        V1, V2 = W1[:, :k1], W2[:, :k2]
        core = np.einsum("tij,ia,jb,tc->cab", A, V1, V2, Q)
        ref = np.einsum("cab,ia,jb,tc->tij", core, V1, V2, Q)
        Ak, err2 = oracle.hosvd(A, k1, k2, Q)
        np.testing.assert_allclose(Ak, ref, atol=1e-11)
        assert err2 == pytest.approx(float(np.sum(A ** 2) - np.sum(core ** 2)), rel=1e-9)


def test_metrics_storage_formulas():
    """Sec. 5.1.2 storage counts and CR."""
    assert oracle.storage_tsvdq(120, 160, 5, 50) == 120 * 5 * 50 + 5 * 160 * 50
    assert oracle.storage_tsvdqII(120, 160, 300) == 300 * 280
    assert oracle.storage_hosvd(10, 20, 30, 2, 3, 4) == 24 + 20 + 60 + 120
    assert oracle.compression_ratio(10, 10, 10, 50, 50) == pytest.approx(10.0)


def test_matched_storage_k2_worked_values():
    """Sec. 5.3 storage equations worked by hand for a hyperspectral-sized case
    (n1 = n2 = 512, n3 = 224, p = 50, k = 20; *Q-SVD budget 20*1024*50 =
    1,024,000 besides Q):
      (n1, k2, p):  k2 (512*50 + 512) <= 1,024,000 - 512^2 = 761,856
                    -> k2 <= 761,856 / 26,112 = 29.18 -> 29
      (k2, k2, p):  50 k2^2 + 1024 k2 <= 1,024,000: k2 = 133 costs 1,020,642,
                    k2 = 134 costs 1,035,016 -> 133"""
    assert oracle.hosvd_matched_k2(512, 512, 224, 50, 20, 0) == 29
    assert oracle.hosvd_matched_k2(512, 512, 224, 50, 20, 1) == 133
    # no feasible k2: the full U1 (n1^2) alone exceeds the budget
    assert oracle.hosvd_matched_k2(512, 512, 224, 1, 1, 0) == 0


def test_matched_storage_k2_is_the_rounded_down_root():
    """The exhaustive search equals the real root of each storage equation,
    rounded down (the paper's 'solve and round down'), clipped to the range."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        n1, n2 = (int(x) for x in rng.integers(4, 300, 2))
        n3 = int(rng.integers(2, 300))
        p = int(rng.integers(1, n3 + 1))
        k = int(rng.integers(1, min(n1, n2) + 1))
        lhs = k * (n1 + n2) * p
        r0 = (lhs - n1 * n1) / (n1 * p + n2)
        b = n1 + n2
        r1 = (-b + math.sqrt(b * b + 4.0 * p * lhs)) / (2.0 * p)
        for variant, root, cap in ((0, r0, n2), (1, r1, min(n1, n2))):
            want = min(cap, math.floor(root + 1e-9)) if root >= 1 else 0
            assert oracle.hosvd_matched_k2(n1, n2, n3, p, k, variant) == want, (n1, n2, n3, p, k)


def test_tiny_config_dct_tsvdq():
    """The tiny config end to end in the oracle: Q = DCT p=4 (Sec. 5.1.1 footnote
    reading), k=3; the error identity holds and sigma match LAPACK per slice."""
    from paper_2409_19402_gb300 import inputs
    A, B = inputs.tiny()
    Q = inputs.dct_q(16, 4)
    np.testing.assert_allclose(Q.astype(np.float64), oracle.dct_q(16, 4), atol=1e-7)
    Uh, s, Vh, Ak, rep = oracle.tsvdq(A, Q, 3)
    # Q is FP32-rounded: Q^T Q = I only to ~1e-7, so the identity holds to ~1e-6
    assert rep.err2 == pytest.approx(rep.discarded2 + rep.proj_err2, rel=1e-5)
    Ah = oracle.mode3(A, Q.astype(np.float64).T)
    for t in range(4):
        np.testing.assert_allclose(s[t], np.linalg.svd(Ah[t], compute_uv=False)[:3], rtol=1e-12)
    C = oracle.qprod(A, B, Q)
    assert C.shape == (16, 32, 20)


def test_qprod_gradient_matches_central_differences():
    """The oracle's analytic gradient of 1/2 |A *Q B - T|^2 (chain rule through
    Def. 3.1) against FP64 central finite differences, on the 16x12x32, p = 8
    instance (B 12 x 10 x 32); the Stiefel gradient is the tangent projection of
    the Euclidean one and is orthogonal to Q's normal space."""
    rng = np.random.default_rng(4)
    n, n1, m, n2, p = 32, 16, 12, 10, 8
    A = rng.standard_normal((n, n1, m)) / 4
    B = rng.standard_normal((n, m, n2)) / 4
    Q = _rand_q(n, p)
    T = rng.standard_normal((n, n1, n2))
    L0, dA, dB, dQE, dQ = oracle.qprod_grad(A, B, Q, T)
    f = lambda A_, B_, Q_: 0.5 * ((oracle.qprod(A_, B_, Q_) - T) ** 2).sum()
    assert L0 == pytest.approx(f(A, B, Q), rel=1e-12)
    # L is quadratic in A and in B (central differences exact up to rounding: large h)
    # and of degree 6 in Q (O(h^2) truncation: small h)
    steps = {"A": 1e-2, "B": 1e-2, "Q": 1e-5}
    for _ in range(12):
        for which, X, dX in (("A", A, dA), ("B", B, dB), ("Q", Q, dQE)):
            h = steps[which]
            idx = tuple(rng.integers(0, s) for s in X.shape)
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            args_p = {"A": (Xp, B, Q), "B": (A, Xp, Q), "Q": (A, B, Xp)}[which]
            args_m = {"A": (Xm, B, Q), "B": (A, Xm, Q), "Q": (A, B, Xm)}[which]
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert fd == pytest.approx(dX[idx], rel=1e-6, abs=1e-8), (which, idx)
    # tangent projection: Q^T dQ is skew-symmetric, and dQ = dQE - Q sym(Q^T dQE)
    S = Q.T @ dQ
    np.testing.assert_allclose(S + S.T, 0.0, atol=1e-10)
    M = Q.T @ dQE
    np.testing.assert_allclose(dQ, dQE - Q @ (0.5 * (M + M.T)), atol=1e-12)


def test_openmp_oracle_build_is_bitwise_the_serial_one():
    """The multi-core baseline build shares out independent slices only: its
    Alg. 4.2 results are bit-identical to the single-thread build's."""
    if not oracle.has_openmp():
        pytest.skip("no OpenMP in this compiler")
    A = RNG.standard_normal((14, 9, 11))
    Q = _rand_q(14, 6)
    a = oracle.tsvdqII(A, Q, 0.9)
    b = oracle.tsvdqII(A, Q, 0.9, omp=True)
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.sig_all, b.sig_all)
    assert np.array_equal(a.Ak, b.Ak) and a.report == b.report
