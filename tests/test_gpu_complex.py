"""Complex transformations (Q in St_{n,p}(C), Sec. 3; the DFT remark after
Def. 3.2) through pprod_c, tsvdq_trunc_c and tsvdqII_c against the complex
FP64 oracle (oracle/complex_q.py, pinned in test_oracle_complex_pins.py).

Tolerances follow the real path's (test_gpu_parity.py): singular values
normwise 1e-5; products elementwise 1e-5 of the Frobenius norm; the error
|A - A_k| within 1e-6 |A| of the oracle's; |A~_k - A_k| <= (1e-6 + ETA g) |A|
with g the largest sigma_R / (sigma_R - sigma_{R+1}) at the kept ranks and
ETA = 2.5e-7 (the FP32 backward error); identical ranks where the oracle's
energy margin certifies them."""
import numpy as np
import pytest
import torch

import oracle
from oracle import complex_q as cq
from paper_2409_19402_gb300 import inputs

pytestmark = pytest.mark.gpu
ETA = 2.5e-7


def _b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_19402_gb300 import binding
    return binding


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def cnorm(x):
    return float(np.sqrt((np.abs(np.asarray(x, dtype=np.complex128)) ** 2).sum()))


def cplx(re, im):
    return re.double().cpu().numpy() + 1j * im.double().cpu().numpy()


def gap(sig, ranks):
    g = 0.0
    for t, R in enumerate(ranks):
        R = int(R)
        if 0 < R < sig.shape[1]:
            d = sig[t, R - 1] - sig[t, R]
            g = max(g, np.inf if d <= 0 else sig[t, R - 1] / d)
    return g


@pytest.mark.parametrize("shape", [(16, 6, 5, 4, 6), (12, 9, 7, 3, 12), (33, 20, 17, 11, 9)])
def test_pprod_c_against_the_oracle(shape):
    n, n1, m, n2, p = shape
    A = inputs.gaussian((n, n1, m), seed=41)
    B = inputs.gaussian((n, m, n2), seed=42)
    Q = inputs.dft_qc(n, p) if p < n else inputs.random_qc(n, p, seed=43)
    b = _b()
    Cr, Ci = b.pprod_c(dev(A), dev(B), dev(Q))
    torch.cuda.synchronize()
    C = cplx(Cr, Ci)
    ref = cq.qprod_c(A, B, Q.astype(np.complex128))
    assert np.abs(C - ref).max() <= 1e-5 * cnorm(ref)


def test_pprod_c_full_dft_is_the_t_product():
    n, n1, m, n2 = 16, 5, 4, 3
    A = inputs.gaussian((n, n1, m), seed=44)
    B = inputs.gaussian((n, m, n2), seed=45)
    b = _b()
    Cr, Ci = b.pprod_c(dev(A), dev(B), dev(inputs.dft_qc(n, n)))
    torch.cuda.synchronize()
    T = cq.tprod(A, B).real / np.sqrt(n)
    scale = cnorm(T)
    assert np.abs(Cr.double().cpu().numpy() - T).max() <= 1e-5 * scale
    assert np.abs(Ci.double().cpu().numpy()).max() <= 1e-5 * scale     # real result


def _check_trunc(A, Q, k):
    b = _b()
    out = b.tsvdq_trunc_c(dev(A), dev(Q), k)
    torch.cuda.synchronize()
    rep = out.report()
    assert rep.status == 0, b.status_str(rep.status)
    U, s, V, Ak, ref = cq.tsvdq_c(A, Q.astype(np.complex128), k)
    full = cq.tsvdq_c(A, Q.astype(np.complex128), min(A.shape[1:]))[1]
    sg = out.s.double().cpu().numpy()
    assert np.linalg.norm(sg - s) <= 1e-5 * np.linalg.norm(s)
    nA = cnorm(A)
    Akg = cplx(*out.Ak)
    assert abs(np.sqrt(max(rep.err2, 0.0)) - np.sqrt(ref.err2)) <= 1e-6 * nA
    g = gap(full, [k] * full.shape[0])
    assert cnorm(Akg - Ak) / nA <= 1e-6 + ETA * g
    assert rep.normA2 == pytest.approx(ref.normA2, rel=1e-5)
    assert rep.normAh2 == pytest.approx(ref.normAh2, rel=1e-5)
    assert rep.discarded2 == pytest.approx(ref.discarded2, rel=1e-4, abs=1e-6 * ref.normA2)
    Ug, Vg = out.Uh.cpu().numpy().astype(np.complex128), out.Vh.cpu().numpy().astype(np.complex128)
    for t in range(Q.shape[1]):                     # factors reproduce each slice's rank-k part
        lhs = (Ug[t] * sg[t]) @ Vg[t].conj().T
        rhs = (U[t] * s[t]) @ V[t].conj().T
        assert np.abs(lhs - rhs).max() <= 2e-5 * max(full[t, 0], 1e-30)
    return out, rep


@pytest.mark.parametrize("case", ["dft_wide", "dft_tall", "random_square", "single"])
def test_tsvdq_trunc_c(case):
    if case == "dft_wide":
        A, Q, k = inputs.gaussian((24, 10, 14), seed=46), inputs.dft_qc(24, 8), 4
    elif case == "dft_tall":
        A, Q, k = inputs.gaussian((20, 17, 9), seed=47), inputs.dft_qc(20, 5), 3
    elif case == "random_square":
        A, Q, k = inputs.gaussian((15, 12, 12), seed=48), inputs.random_qc(15, 15, seed=49), 12
    else:
        A, Q, k = inputs.gaussian((1, 5, 3), seed=50), np.ones((1, 1), np.complex64), 1
    _check_trunc(A, Q, k)


def _check_II(A, Q, gamma):
    b = _b()
    out = b.tsvdqII_c(dev(A), dev(Q), gamma)
    torch.cuda.synchronize()
    rep = out.report()
    assert rep.status == 0, b.status_str(rep.status)
    rho, U, s, V, Ak, sig, ref = cq.tsvdqII_c(A, Q.astype(np.complex128), gamma)
    # certified ranks: the oracle's energy margin exceeds the sigma perturbation
    keys = np.sort((sig ** 2).ravel())[::-1]
    c = np.cumsum(keys)
    K = ref.K
    margin = min(c[K - 1] - gamma * c[-1], gamma * c[-1] - (c[K - 2] if K >= 2 else 0.0)) / c[-1]
    full = b.tsvdq_trunc_c(dev(A), dev(Q), min(A.shape[1:]), want_ak=False)
    torch.cuda.synchronize()
    sg_all = full.s.double().cpu().numpy()
    assert np.linalg.norm(sg_all - sig) <= 1e-5 * np.linalg.norm(sig)
    pert = np.abs(np.sort((sg_all ** 2).ravel())[::-1] - keys).sum() / keys.sum()
    if gamma < 1.0:
        assert margin > 4 * pert, (margin, pert)
    assert rep.K == K and np.array_equal(out.rho.cpu().numpy(), rho)
    nA = cnorm(A)
    assert abs(np.sqrt(max(rep.err2, 0.0)) - np.sqrt(ref.err2)) <= 1e-6 * nA
    assert cnorm(cplx(*out.Ak) - Ak) / nA <= 1e-6 + ETA * gap(sig, rho)
    for t, (Ut, st, Vt) in enumerate(out.slices()):
        if len(st) == 0:
            continue
        Ut, Vt = Ut.numpy().astype(np.complex128), Vt.numpy().astype(np.complex128)
        lhs = (Ut * st.numpy()) @ Vt.conj().T
        rhs = (U[t] * s[t]) @ V[t].conj().T
        assert np.abs(lhs - rhs).max() <= 2e-5 * sig[t, 0]
    return out, rep, ref


@pytest.mark.parametrize("gamma", [0.5, 0.9, 0.99])
def test_tsvdqII_c_small(gamma):
    _check_II(inputs.gaussian((30, 14, 19), seed=51), inputs.dft_qc(30, 10), gamma)


def test_tsvdqII_c_video_dft_p50():
    """The video workload with the DFT rows as Q (p = 50)."""
    A = inputs.video()
    _, rep, ref = _check_II(A, inputs.dft_qc(300, 50), 0.99)
    assert rep.kappa == ref.kappa


def test_real_q_through_the_complex_path_matches_the_real_path():
    b = _b()
    A = inputs.gaussian((18, 11, 13), seed=52)
    Qr = inputs.random_q(18, 6, seed=53)
    oc = b.tsvdqII_c(dev(A), dev(Qr.astype(np.complex64)), 0.9)
    orr = b.tsvdqII(dev(A), dev(Qr), 0.9)
    torch.cuda.synchronize()
    assert np.array_equal(oc.rho.cpu().numpy(), orr.rho.cpu().numpy())
    Akc = cplx(*oc.Ak)
    Akr = orr.Ak.double().cpu().numpy()
    nA = cnorm(A)
    assert cnorm(Akc - Akr) / nA <= 1e-5
    assert np.abs(Akc.imag).max() <= 1e-5 * nA


def test_complex_status_and_shape_errors():
    b = _b()
    A = dev(inputs.gaussian((8, 6, 5), seed=54))
    Q = inputs.dft_qc(8, 4)
    Qbad = Q.copy()
    Qbad[:, 0] *= 2.0
    out = b.tsvdqII_c(A, dev(Qbad), 0.9, check_q=True)
    torch.cuda.synchronize()
    assert out.report().status == b.PP_ENOTORTHO
    with pytest.raises(b.PPError):
        b.tsvdqII_c(dev(inputs.gaussian((4, 400, 400), seed=55)), dev(inputs.dft_qc(4, 2)), 0.9)
