"""tsvdqII_noalloc: the *Q-SVDII entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or allocation is
forbidden after start-up because it can synchronise the device).  It takes no
workspace argument and runs on the library's fixed device scratch array.

Checked through the C ABI against the existing tsvdqII (which takes a
caller-allocated workspace), on two calls in a row with different shapes, with
the tolerances of the parity tests; then a shape whose workspace exceeds the
fixed scratch must be rejected before anything runs.  This file is collected
last so that a failure here cannot hide the results of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_19402_gb300 import inputs

pytestmark = pytest.mark.gpu


def _b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_19402_gb300 import binding
    return binding


def _norm(t):
    return float(t.double().norm())


def _compare(b, A, Q, gamma):
    Ad, Qd = torch.from_numpy(A).cuda(), torch.from_numpy(Q).cuda()
    ref = b.tsvdqII(Ad, Qd, gamma)
    got = b.tsvdqII_noalloc(Ad, Qd, gamma)
    torch.cuda.synchronize()
    r_ref, r_got = ref.report(), got.report()
    assert r_got.status == 0, b.status_str(r_got.status)
    assert r_got.K == r_ref.K and r_got.kappa == r_ref.kappa
    assert torch.equal(got.rho, ref.rho) and torch.equal(got.offs, ref.offs)
    nA = _norm(Ad)
    assert _norm(got.Ak - ref.Ak) <= 1e-6 * nA
    kappa = int(r_ref.kappa)
    l, m = A.shape[1], A.shape[2]
    s_ref, s_got = ref.s[:kappa].double(), got.s[:kappa].double()
    assert float((s_got - s_ref).norm()) <= 1e-5 * float(s_ref.norm())
    for (Ur, sr, Vr), (Ug, sg, Vg) in zip(ref.slices(), got.slices()):
        if len(sr):
            dr = (Ur.double() * sr.double()) @ Vr.double().T
            dg = (Ug.double() * sg.double()) @ Vg.double().T
            assert float((dg - dr).norm()) <= 1e-6 * nA
    assert abs(r_got.err2 - r_ref.err2) <= 1e-6 * r_ref.normA2
    return got


def test_noalloc_matches_tsvdqII_two_calls_in_a_row():
    b = _b()
    A1, _ = inputs.tiny()
    _compare(b, A1, inputs.dct_q(16, 4), 0.8)                       # first call: set-up
    A2 = inputs.gaussian((45, 37, 53), seed=21)
    _compare(b, A2, inputs.random_q(45, 7, seed=22), 0.9)           # second call, other shape
    # a third call allocates nothing on the device
    free0, _ = torch.cuda.mem_get_info()
    _compare(b, A1, inputs.dct_q(16, 4), 0.8)
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1


def test_noalloc_video_workload_fits():
    b = _b()
    A = inputs.video()
    _compare(b, A, inputs.u3_q(A, 50), 0.99)


def test_noalloc_rejects_shapes_beyond_the_scratch():
    b = _b()
    need = b.workspace_bytes(b.PP_OP_TSVDQII, l=120, m=160, n=300, p=300)
    assert need > 16 * 1024 * 1024
    fake = ctypes.c_void_p(1 << 20)          # never dereferenced: rejected on the host
    st = b.lib().tsvdqII_noalloc(fake, fake, 120, 160, 300, 300, 0.99, fake, fake, fake, fake,
                                 fake, None, None, None, None)
    assert st == b.PP_EWORKSPACE
