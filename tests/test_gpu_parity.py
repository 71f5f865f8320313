"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded FP32 inputs.

Tolerances (what the accuracy of the method's FP32 results supports):
  * mode-3 products (tensor cores, 3-pass split TF32): per entry
    |y~ - y| <= (2 S + 16) u sum_s |M(t,s)| |X(s)|, u = 2^-24, S terms: the
    split drops at most 3 * 2^-22 = 12 u of each product, and S u per sum is
    doubled because the tensor core does not round to nearest;
  * facewise products (the same tensor-core 3-pass split, S = m terms):
    (2 S + 16) u sum_s |A(i,s)| |B(s,j)|;
  * singular values: normwise |s~ - s|_2 <= 1e-5 |s|_2 over every slice;
  * reconstruction: | |A - A~_k| - |A - A_k| | <= 1e-6 |A| (the stated bar), and
    |A~_k - A_k|_F <= (1e-6 + ETA g) |A| where g = max_t sigma_{t,R}/(sigma_{t,R} -
    sigma_{t,R+1}) is the gap condition of the truncation: the best rank-R
    approximation moves by about |E| sigma_R/gap under a perturbation E, and
    the relative backward error of the FP32 path is ETA = 2.5e-7 (the mode-3
    product alone measures 2.5e-7 in Frobenius norm on Gaussian data);
  * ranks (Alg. 4.2): identical K and rho, with the oracle's margin
    certified against the singular-value discrepancy;
  * the selection itself is bit-exact: the oracle's Alg. 4.2 steps 4-7 run on
    the GPU's own singular values reproduce the GPU's K and rho exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_19402_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
ETA = 2.5e-7     # relative backward error of the FP32 path (see the module docstring)


def _b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_19402_gb300 import binding
    return binding


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f64(x):
    return np.asarray(x, dtype=np.float64)


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("shape", [(16, 32, 24, 4), (45, 37, 29, 7), (300, 120, 160, 50),
                                   (9, 1, 1, 9), (64, 3, 130, 1)])
def test_mode3_projection_and_back(shape):
    """Def. 2.2 both ways (Q^T: n -> p, Q: p -> n), elementwise within the FP32 bound."""
    b = _b()
    n, l, m, p = shape
    X = inputs.gaussian((n, l, m), seed=n + p)
    Q = inputs.random_q(n, p, seed=7)
    Y = host(b.pprod_mode3(dev(X), dev(Q), 0))
    ref = oracle.mode3(X, f64(Q).T)
    bound = (2 * n + 16) * U32 * oracle.mode3(np.abs(f64(X)), np.abs(f64(Q)).T)
    assert np.all(np.abs(Y - ref) <= bound + 1e-30)
    Xh = inputs.gaussian((p, l, m), seed=3 * n + p)
    Z = host(b.pprod_mode3(dev(Xh), dev(Q), 1))
    ref2 = oracle.mode3(Xh, f64(Q))
    bound2 = (2 * p + 16) * U32 * oracle.mode3(np.abs(f64(Xh)), np.abs(f64(Q)))
    assert np.all(np.abs(Z - ref2) <= bound2 + 1e-30)


@pytest.mark.parametrize("shape", [(4, 32, 24, 20), (3, 70, 33, 129), (1, 1, 1, 1), (8, 256, 256, 64)])
def test_facewise_product(shape):
    """Def. 2.3, elementwise within the bound of the 3-pass split tf32 product."""
    b = _b()
    p, n1, m, n2 = shape
    A = inputs.gaussian((p, n1, m), seed=1)
    B = inputs.gaussian((p, m, n2), seed=2)
    C = host(b.pprod_facewise(dev(A), dev(B)))
    ref = oracle.facewise(A, B)
    bound = (2 * m + 16) * U32 * oracle.facewise(np.abs(f64(A)), np.abs(f64(B)))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)


def test_pprod_tiny_config():
    """Def. 3.1 on the tiny config (A 32x24x16, B 24x20x16, DCT p=4)."""
    b = _b()
    A, B = inputs.tiny()
    Q = inputs.dct_q(16, 4)
    C = host(b.pprod(dev(A), dev(B), dev(Q)))
    ref = oracle.qprod(A, B, Q)
    scale = np.abs(oracle.qprod(np.abs(f64(A)), np.abs(f64(B)), np.abs(f64(Q))))
    assert np.abs(C - ref).max() <= 1e-5 * scale.max()


def test_pprod_p_equals_n_is_starM():
    """p = n with orthogonal Q: the same kernels compute A *M B with M = Q^T."""
    b = _b()
    n = 12
    A = inputs.gaussian((n, 9, 7), seed=4)
    B = inputs.gaussian((n, 7, 5), seed=5)
    Q = inputs.random_q(n, n, seed=6)
    C = host(b.pprod(dev(A), dev(B), dev(Q)))
    ref = oracle.mprod(A, B, f64(Q).T, f64(Q))
    assert np.abs(C - ref).max() <= 1e-5 * np.abs(ref).max()


# ------------------------------------------------------------------ decompositions
def _norm(x):
    return float(np.sqrt((f64(x) ** 2).sum()))


def gap_condition(sig_all, ranks):
    """max over slices of sigma_R / (sigma_R - sigma_{R+1}) at the kept rank R."""
    g = 0.0
    for t, R in enumerate(ranks):
        R = int(R)
        if 0 < R < sig_all.shape[1]:
            d = sig_all[t, R - 1] - sig_all[t, R]
            g = max(g, np.inf if d <= 0 else sig_all[t, R - 1] / d)
    return g


def _check_recon(Ak_gpu, err2_gpu, Ak_ref, err2_ref, A, sig_all, ranks):
    nA = _norm(A)
    assert abs(np.sqrt(max(err2_gpu, 0.0)) - np.sqrt(err2_ref)) <= 1e-6 * nA
    g = gap_condition(sig_all, ranks)
    rel = _norm(Ak_gpu - Ak_ref) / nA
    assert rel <= 1e-6 + ETA * g, (rel, g)


@pytest.mark.parametrize("case", [
    ("tiny", 3), ("tall", 5), ("odd", 23), ("ragged", 4), ("single", 1)])
def test_tsvdq_trunc(case):
    """Alg. 4.1 against the oracle: sigma, A_k, error terms (Thm. 4.2)."""
    b = _b()
    name, k = case
    if name == "tiny":
        A, _ = inputs.tiny()
        Q = inputs.dct_q(16, 4)
    elif name == "tall":
        A = inputs.gaussian((10, 40, 24), seed=11)      # l > m: vectors are columns
        Q = inputs.random_q(10, 5, seed=12)
    elif name == "odd":
        A = inputs.gaussian((9, 23, 31), seed=13)       # odd b, k = b, p = n (*M form)
        Q = inputs.random_q(9, 9, seed=14)
    elif name == "ragged":
        A = inputs.gaussian((45, 37, 53), seed=15)
        Q = inputs.random_q(45, 7, seed=16)
    else:
        A = inputs.gaussian((1, 5, 3), seed=17)          # n = p = 1
        Q = np.ones((1, 1), dtype=np.float32)
    out = b.tsvdq_trunc(dev(A), dev(Q), k)
    torch.cuda.synchronize()
    rep = out.report()
    assert rep.status == 0, b.status_str(rep.status)
    Uh, s, Vh, Ak, ref = oracle.tsvdq(A, Q, k)
    sg = host(out.s)
    assert np.linalg.norm(sg - s) <= 1e-5 * np.linalg.norm(s)
    sig_all = np.stack([oracle.svd(x)[1] for x in oracle.mode3(A, f64(Q).T)])
    _check_recon(host(out.Ak), rep.err2, Ak, ref.err2, A, sig_all, [k] * Q.shape[1])
    assert rep.discarded2 == pytest.approx(ref.discarded2, rel=1e-5, abs=1e-6 * ref.normA2)
    # energies: FP32 partial sums over <= 16 terms, combined in FP64 (<= 16 u relative)
    assert rep.normA2 == pytest.approx(ref.normA2, rel=16 * U32)
    assert rep.kappa == k * Q.shape[1] and rep.K == 0
    # factors: orthonormal columns and sigma_q u_q v_q^T matches per slice
    U, V = host(out.Uh), host(out.Vh)
    for t in range(Q.shape[1]):
        nz = sg[t] > 1e-6 * sg[t, 0]
        Ut, Vt = U[t][:, nz], V[t][:, nz]
        assert np.abs(Ut.T @ Ut - np.eye(nz.sum())).max() < 1e-4
        assert np.abs(Vt.T @ Vt - np.eye(nz.sum())).max() < 1e-4
        np.testing.assert_allclose((U[t] * sg[t]) @ V[t].T, (Uh[t] * s[t]) @ Vh[t].T,
                                   atol=1e-5 * max(s[t, 0], 1e-30))


def _margin(sig_ref, gamma, K):
    """Oracle margin of the K decision: min(c_K - gamma c_N, gamma c_N - c_{K-1}) / c_N."""
    keys = np.sort((sig_ref ** 2).ravel())[::-1]
    c = np.cumsum(keys)
    cN = c[-1]
    lo = c[K - 2] if K >= 2 else 0.0
    return min(c[K - 1] - gamma * cN, gamma * cN - lo) / cN, keys


def _tsvdqII_case(A, Q, gamma, oracle_omp=False, **opts):
    b = _b()
    out = b.tsvdqII(dev(A), dev(Q), gamma, **opts)
    full = b.tsvdq_trunc(dev(A), dev(Q), min(A.shape[1], A.shape[2]), want_ak=False, **opts)
    torch.cuda.synchronize()
    rep = out.report()
    assert rep.status == 0, b.status_str(rep.status)
    ref = oracle.tsvdqII(A, Q, gamma, omp=oracle_omp and oracle.has_openmp())
    sig_gpu = host(full.s)                                   # every singular value
    # (1) bit-exact selection on the GPU's own singular values
    K2, rho2, kept2, total2 = oracle.select_energy(sig_gpu, gamma)
    rho = out.rho.cpu().numpy()
    assert rep.K == K2 and np.array_equal(rho, rho2)
    offs = out.offs.cpu().numpy()
    assert offs[0] == 0 and np.array_equal(np.diff(offs), rho) and offs[-1] == rep.kappa
    # (2) singular values, normwise
    assert np.linalg.norm(sig_gpu - ref.sig_all) <= 1e-5 * np.linalg.norm(ref.sig_all)
    # (3) identical ranks, certified: prefix sums move by at most sum |d sigma^2|
    #     (gamma = 1 keeps every value that still changes the FP64 total: no margin)
    if ref.report.K > 0 and gamma < 1.0:
        margin, keys = _margin(ref.sig_all, gamma, ref.report.K)
        pert = np.abs(np.sort((sig_gpu ** 2).ravel())[::-1] - keys).sum() / keys.sum()
        assert margin > 4 * pert, f"seed not certifiable: margin {margin:.3e} vs {pert:.3e}"
    assert rep.K == ref.report.K
    assert np.array_equal(rho, ref.rho)
    # (4) reconstruction and error terms (Thm. 4.4)
    _check_recon(host(out.Ak), rep.err2, ref.Ak, ref.report.err2, A, ref.sig_all, ref.rho)
    assert rep.discarded2 == pytest.approx(ref.report.discarded2, rel=1e-4,
                                           abs=1e-6 * ref.report.normA2)
    # (5) packed factors reproduce sigma_q u_q v_q^T slice by slice
    for t, (Ut, st, Vt) in enumerate(out.slices()):
        Ut, st, Vt = f64(Ut), f64(st), f64(Vt)
        if len(st) == 0:
            continue
        np.testing.assert_allclose((Ut * st) @ Vt.T, (ref.Uh[t] * ref.s[t]) @ ref.Vh[t].T,
                                   atol=2e-5 * ref.sig_all[t, 0])
    return rep, ref


@pytest.mark.parametrize("precond", [True, False])
@pytest.mark.parametrize("shape", [(40, 23, 57), (40, 57, 23), (24, 33, 33), (64, 130, 9),
                                   (16, 37, 300), (14, 130, 176), (12, 128, 176), (12, 176, 128),
                                   (12, 100, 177)])
def test_tsvdqII_with_and_without_qr_preconditioner(shape, precond):
    """Both Jacobi paths (rows of R from the QR with column pivoting, or the
    slice itself) against the oracle, on wide, tall, square and very flat slices.
    The first four (and the video-shaped slices) take the register-resident QR,
    128 x 176 and 176 x 128 at its largest shape (128 vectors of 176 entries,
    11 float4 per lane); 37 x 300 (vectors longer than 176), 100 x 177 (just
    past that bound) and 130 x 176 (more than 128 vectors) take the
    shared-memory QR."""
    n, l, m = shape
    A = inputs.gaussian(shape, seed=31 + l)
    Q = inputs.random_q(n, 12, seed=32)
    _tsvdqII_case(A, Q, 0.9, precond=precond)


def test_tsvdqII_tiny():
    A, _ = inputs.tiny()
    _tsvdqII_case(A, inputs.dct_q(16, 4), 0.8)


@pytest.mark.parametrize("gamma", [0.5, 0.9, 1.0])
def test_tsvdqII_ragged_shapes(gamma):
    A = inputs.gaussian((45, 37, 53), seed=21)
    _tsvdqII_case(A, inputs.random_q(45, 7, seed=22), gamma)


def test_tsvdqII_many_slices_single_cta_path():
    """p >= 76 slices: one CTA per slice (no cluster split)."""
    A = inputs.gaussian((100, 20, 30), seed=25)
    _tsvdqII_case(A, inputs.random_q(100, 80, seed=26), 0.9)


def test_tsvdqII_tall_slices():
    A = inputs.gaussian((20, 48, 30), seed=23)
    _tsvdqII_case(A, inputs.random_q(20, 6, seed=24), 0.95)


def test_tsvdqII_video_p50():
    """Video-shaped config: 120x160x300, Q = U3 with p = 50, gamma = 0.99."""
    A = inputs.video()
    rep, ref = _tsvdqII_case(A, inputs.u3_q(A, 50), 0.99)
    assert rep.sweeps <= 30


@pytest.mark.slow
def test_tsvdqII_video_p_equals_n():
    """The invertible *M comparison of the video config: p = n = 300, full U3."""
    A = inputs.video()
    _tsvdqII_case(A, inputs.u3_q(A, 300), 0.99)


@pytest.mark.parametrize("shape", [(12, 256, 300), (10, 200, 130)])
def test_blocked_jacobi_large_slices(shape):
    """Slices that exceed shared memory take the block-cyclic Jacobi path
    (256 x 300: rows are the vectors; 200 x 130: columns are)."""
    A = inputs.gaussian(shape, seed=31)
    _tsvdqII_case(A, inputs.random_q(shape[0], 3, seed=32), 0.9)


# ------------------------------------------------------------------ degenerate inputs
def test_zero_tensor():
    b = _b()
    A = np.zeros((6, 5, 7), dtype=np.float32)
    Q = inputs.random_q(6, 3, seed=1)
    out = b.tsvdqII(dev(A), dev(Q), 0.9)
    tr = b.tsvdq_trunc(dev(A), dev(Q), 2)
    torch.cuda.synchronize()
    rep = out.report()
    assert rep.status == 0 and rep.K == 0 and rep.kappa == 0
    assert np.all(out.rho.cpu().numpy() == 0)
    assert np.all(host(out.Ak) == 0)
    assert np.all(host(tr.s) == 0) and np.all(host(tr.Uh) == 0) and np.all(host(tr.Vh) == 0)


def test_rank_deficient_slices():
    """Exactly rank-2 transform-domain slices: sigma beyond 2 vanish, A_k exact at k = 2."""
    b = _b()
    n, l, m, p = 8, 20, 16, 4
    rng = np.random.default_rng(5)
    Q = inputs.random_q(n, p, seed=9)
    Ah = np.stack([rng.standard_normal((l, 2)) @ rng.standard_normal((2, m)) for _ in range(p)])
    A = oracle.mode3(Ah, f64(Q)).astype(np.float32)          # lies in range(Q)
    out = b.tsvdq_trunc(dev(A), dev(Q), 3)
    torch.cuda.synchronize()
    rep = out.report()
    s = host(out.s)
    assert np.all(s[:, 2] <= 1e-5 * s[:, 0])
    assert rep.err2 <= 1e-10 * rep.normA2


def test_device_error_statuses():
    """Device-detected conditions land in pp_report.status (no fault, no trap)."""
    b = _b()
    A = inputs.gaussian((10, 12, 14), seed=2)
    Q = inputs.random_q(10, 4, seed=3)
    Qbad = (2.0 * Q).astype(np.float32)
    rep = b.tsvdq_trunc(dev(A), dev(Qbad), 2, check_q=True).report()
    assert rep.status == b.PP_ENOTORTHO
    An = A.copy()
    An[3, 4, 5] = np.nan
    rep = b.tsvdq_trunc(dev(An), dev(Q), 2, check_finite=True).report()
    assert rep.status == b.PP_ENONFINITE
    rep = b.tsvdq_trunc(dev(A), dev(Q), 2, max_sweeps=1).report()
    assert rep.status == b.PP_ENOCONV
    rep = b.tsvdq_trunc(dev(A), dev(Q), 2, check_q=True, check_finite=True).report()
    assert rep.status == 0


def test_deterministic():
    b = _b()
    A = inputs.gaussian((30, 40, 50), seed=8)
    Q = inputs.random_q(30, 6, seed=9)
    o1 = b.tsvdqII(dev(A), dev(Q), 0.9)
    o2 = b.tsvdqII(dev(A), dev(Q), 0.9)
    torch.cuda.synchronize()
    assert torch.equal(o1.Ak, o2.Ak) and torch.equal(o1.rho, o2.rho)
    assert bytes(o1.rep.cpu().numpy()) == bytes(o2.rep.cpu().numpy())
