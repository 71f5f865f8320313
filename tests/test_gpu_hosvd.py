"""hosvd_compare against the oracle: truncated HOSVD (k1, k2, p) with the mode-3
factor U3 = Q (Sec. 4.2) and the *Q-SVD with k = min(k1, k2), whose error is no
larger (Thm. 4.6).  Tolerance: the reconstruction bar | |A - A~| - |A - A| | <=
1e-6 |A| on both errors (second order in the factor subspaces, so no gap term)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_19402_gb300 import inputs

pytestmark = pytest.mark.gpu


def _b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_19402_gb300 import binding
    return binding


def _case(A, p, k1, k2):
    b = _b()
    Q = inputs.u3_q(A, p)
    Ad, Qd = torch.from_numpy(A).cuda(), torch.from_numpy(Q).cuda()
    rep, Ak = b.hosvd_compare(Ad, Qd, k1, k2, want_ak=True)
    assert rep.status == 0, b.status_str(rep.status)
    nA = float(np.sqrt((A.astype(np.float64) ** 2).sum()))
    Ak_ref, e_hos = oracle.hosvd(A, k1, k2, Q)
    _, _, _, _, r_q = oracle.tsvdq(A, Q, min(k1, k2))
    assert abs(np.sqrt(rep.err2_hosvd) - np.sqrt(e_hos)) <= 1e-6 * nA
    assert abs(np.sqrt(rep.err2_tsvdq) - np.sqrt(r_q.err2)) <= 1e-6 * nA
    assert rep.err2_tsvdq <= rep.err2_hosvd * (1 + 1e-6)            # Thm. 4.6
    # the returned A_(k1,k2,p) reproduces the reported error
    e_direct = float(((Ak.double() - Ad.double()) ** 2).sum())
    assert e_direct == pytest.approx(rep.err2_hosvd, rel=1e-5)
    assert rep.k == min(k1, k2) and rep.k1 == k1 and rep.k2 == k2
    return rep


def test_hosvd_small_lowrank_plus_noise():
    rng = np.random.default_rng(7)
    core = rng.standard_normal((20, 4, 4)).astype(np.float64)
    A = np.einsum("tab,ia,jb->tij", core, rng.standard_normal((12, 4)), rng.standard_normal((16, 4)))
    A = (A + 0.05 * rng.standard_normal(A.shape)).astype(np.float32)
    _case(A, 6, 5, 7)


def test_hosvd_video_shaped():
    A = inputs.video()
    for k1, k2 in [(20, 30), (40, 40)]:
        _case(A, 50, k1, k2)


def test_hosvd_hyperspectral_shaped_reduced():
    A = inputs.hyperspectral(l=128, m=128, n=224)
    _case(A, 10, 20, 20)


def test_section_5_3_comparison_pipeline_on_the_gpu():
    """The Sec. 5.3 protocol end to end on the device: Q = U3 from pprod_u3, the
    *Q-SVD with truncation k, the *Q-SVDII energy gamma = kept / |A-hat|^2 taken
    from that run (no worse, Thm. 4.5), and the HOSVD (k2, k2, p) with k2 from
    the storage equations (no more storage than the *Q-SVD), whose error matches
    the oracle's HOSVD at the same k2."""
    b = _b()
    A = inputs.hyperspectral(l=128, m=128, n=224)
    n, l, m = A.shape
    p, k = 25, 5
    Ad = torch.from_numpy(A).cuda()
    Qd, _, _ = b.pprod_u3(Ad, p)
    tq = b.tsvdq_trunc(Ad, Qd, k)
    r1 = tq.report()
    assert r1.status == 0
    gamma = r1.kept2 / r1.normAh2
    r2 = b.tsvdqII(Ad, Qd, gamma).report()
    assert r2.status == 0
    assert r2.err2 <= r1.err2 * (1 + 1e-5)                           # Thm. 4.5
    assert oracle.storage_tsvdqII(l, m, r2.kappa) <= oracle.storage_tsvdq(l, m, k, p)
    k2 = b.hosvd_matched_k2(l, m, n, p, k, 1)
    assert k2 >= 1
    assert (oracle.storage_hosvd(l, m, n, k2, k2, p)
            <= oracle.storage_tsvdq(l, m, k, p) + n * p)
    rep, _ = b.hosvd_compare(Ad, Qd, k2, k2)
    assert rep.status == 0
    Q = Qd.cpu().numpy()
    _, e_hos = oracle.hosvd(A, k2, k2, Q)
    nA = float(np.sqrt((A.astype(np.float64) ** 2).sum()))
    assert abs(np.sqrt(rep.err2_hosvd) - np.sqrt(e_hos)) <= 1e-6 * nA
