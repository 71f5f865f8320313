"""CPU-only checks of the C ABI: the library loads, exports every function
declared in include/pprod.h, and rejects bad arguments on the host before any
CUDA call is made (no GPU is touched here)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pprod.h")


def _lib():
    from paper_2409_19402_gb300 import binding
    import __graft_entry__
    if not os.path.exists(binding.LIB_PATH):
        __graft_entry__.build()
    return binding


def declared_functions():
    txt = open(HEADER).read()
    return re.findall(r"PP_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)


def test_header_declares_the_entry_points():
    names = set(declared_functions())
    for f in ("pprod_mode3", "pprod_facewise", "pprod", "tsvdq_trunc", "tsvdqII",
              "pp_workspace_bytes", "pp_status_str", "pp_version"):
        assert f in names


def test_library_exports_every_declared_symbol():
    b = _lib()
    L = b.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings_and_version():
    b = _lib()
    assert b.status_str(0) == "PP_OK"
    for s in range(1, 10):
        assert b.status_str(s).startswith("PP_E")
    assert "sm_103a" in b.version()


def test_workspace_sizes():
    b = _lib()
    w1 = b.workspace_bytes(b.PP_OP_TSVDQ, l=120, m=160, n=300, p=50, k=5)
    w2 = b.workspace_bytes(b.PP_OP_TSVDQII, l=120, m=160, n=300, p=50)
    w3 = b.workspace_bytes(b.PP_OP_TSVDQII, l=120, m=160, n=300, p=300)
    assert 0 < w1 <= w2 < w3
    assert w2 >= 2 * 50 * 120 * 160 * 4            # A-hat and its rebuild at least
    assert b.workspace_bytes(b.PP_OP_MODE3, l=4, m=4, n=4, p=2) == 0
    assert b.workspace_bytes(b.PP_OP_TSVDQ, l=4, m=4, n=2, p=3) == 0   # p > n: invalid
    assert b.workspace_bytes(b.PP_OP_PPROD, l=4, m=5, n=6, p=2, n2=3) >= 4 * (2 * 20 + 2 * 15 + 2 * 12)


def _img(P, S, faces=1):
    """tf32 operand image of P x S per face: one 32 KB block (hi and lo of two
    32-term chunks) per 64-row tile and 64-term stage."""
    return faces * ((P + 63) // 64) * ((S + 63) // 64) * 32768


def test_projected_product_workspace_holds_the_operand_images():
    """pprod's workspace: the transform-domain tensors, the Q^T and Q images and
    the facewise operands' images, the last capped at 32 MB (faces beyond run in
    groups); host arithmetic only."""
    b = _lib()
    ws = lambda n1, m, n2, n, p: b.workspace_bytes(b.PP_OP_PPROD, l=n1, m=m, n=n, p=p, n2=n2)
    # differentiation workload: 64 faces of 256 x 256 by 256 x 64 (the 64-wide
    # side is the image's row side), 8 MB of facewise image
    n1, m, n2, n, p = 256, 256, 64, 512, 64
    tensors = 4 * p * (n1 * m + m * n2 + n1 * n2)
    assert ws(n1, m, n2, n, p) >= tensors + _img(p, n) + _img(n, p) + _img(64, m, p)
    # 1 MB images per face (8 x 2048 by 2048 x 4): 40 and 80 faces both exceed
    # the cap, so doubling p adds only the tensors and the Q images
    n1, m, n2, n = 8, 2048, 4, 96
    grow = ws(n1, m, n2, n, 80) - ws(n1, m, n2, n, 40)
    expect = (4 * 40 * (n1 * m + m * n2 + n1 * n2) + _img(80, n) - _img(40, n)
              + _img(n, 80) - _img(n, 40))
    assert grow == expect
    # below the cap the region grows with the faces: 16 -> 24 faces adds 8 images
    grow = ws(n1, m, n2, n, 24) - ws(n1, m, n2, n, 16)
    expect = (4 * 8 * (n1 * m + m * n2 + n1 * n2) + _img(24, n) - _img(16, n)
              + _img(n, 24) - _img(n, 16) + _img(4, m, 8))
    assert grow == expect


FAKE = ctypes.c_void_p(1 << 20)     # never dereferenced: the host rejects first


def test_host_validation_codes():
    b = _lib()
    L = b.lib()
    # NULL pointers -> PP_EINVAL
    assert L.pprod_mode3(None, 4, 4, 4, None, 2, 0, None, None) == b.PP_EINVAL
    # bad transpose flag
    assert L.pprod_mode3(FAKE, 4, 4, 4, FAKE, 2, 7, FAKE, None) == b.PP_EINVAL
    # p > n
    assert L.pprod_mode3(FAKE, 4, 4, 4, FAKE, 5, 0, FAKE, None) == b.PP_ESHAPE
    # k out of range
    o = b.pp_opts()
    for k in (0, 5):
        assert L.tsvdq_trunc(FAKE, FAKE, 4, 6, 8, 2, k, FAKE, FAKE, FAKE, None, None,
                             ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_ESHAPE
    # workspace too small / misaligned / missing
    assert L.tsvdq_trunc(FAKE, FAKE, 4, 6, 8, 2, 2, FAKE, FAKE, FAKE, None, None,
                         ctypes.byref(o), FAKE, 16, None) == b.PP_EWORKSPACE
    assert L.tsvdq_trunc(FAKE, FAKE, 4, 6, 8, 2, 2, FAKE, FAKE, FAKE, None, None,
                         ctypes.byref(o), ctypes.c_void_p((1 << 20) + 4), 1 << 30,
                         None) == b.PP_EWORKSPACE
    assert L.tsvdq_trunc(FAKE, FAKE, 4, 6, 8, 2, 2, FAKE, FAKE, FAKE, None, None,
                         ctypes.byref(o), None, 0, None) == b.PP_EWORKSPACE
    # gamma outside (0, 1]
    for g in (0.0, -0.5, 1.0000001, float("nan")):
        assert L.tsvdqII(FAKE, FAKE, 4, 6, 8, 2, g, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                         ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_EINVAL
    # slice longer than the Jacobi kernel is built for
    assert L.tsvdqII(FAKE, FAKE, 4, 4096, 8, 2, 0.9, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                     ctypes.byref(o), FAKE, 1 << 40, None) == b.PP_ENOSYS
    # facewise / pprod shapes
    assert L.pprod_facewise(FAKE, FAKE, 0, 3, 3, 2, FAKE, None) == b.PP_ESHAPE
    assert L.pprod(FAKE, FAKE, FAKE, 3, 3, 3, 4, 5, FAKE, FAKE, 1 << 20, None) == b.PP_ESHAPE


def test_binding_refuses_cpu_tensors():
    import torch
    b = _lib()
    with pytest.raises(ValueError):
        b.pprod_mode3(torch.zeros(4, 2, 2), torch.zeros(4, 2), 0)


def test_jacobi_shape_registration_validates_on_host():
    b = _lib()
    L = b.lib()
    assert L.pp_set_jacobi_shape(120, 160, 50, 9, 16) == b.PP_EINVAL     # C > 8
    assert L.pp_set_jacobi_shape(120, 160, 50, 3, 12) == b.PP_EINVAL     # GW not 8/16/32
    assert L.pp_set_jacobi_shape(0, 160, 50, 3, 16) == b.PP_EINVAL
    assert L.pp_set_jacobi_shape(120, 160, 50, 5, 16) == b.PP_OK
    assert L.pp_set_jacobi_shape(120, 160, 50, 0, 0) == b.PP_OK          # removal


def test_autotune_candidates():
    from paper_2409_19402_gb300 import autotune
    c = autotune.candidates(120, 160)
    assert (1, 16) in c and (5, 16) in c and (8, 32) in c
    assert all(C == 1 or 120 >= 4 * C for C, _ in c)
    assert autotune.candidates(6, 9) == [(1, 16)]


def test_matched_storage_k2_matches_the_oracle_search():
    """pp_hosvd_matched_k2 (closed form, host) equals the oracle's exhaustive
    search over k2 on a grid of shapes, including the infeasible cases."""
    import numpy as np
    import oracle
    b = _lib()
    rng = np.random.default_rng(12)
    cases = [(512, 512, 224, 50, 20), (120, 160, 300, 50, 5), (512, 512, 224, 1, 1),
             (32, 24, 16, 4, 3), (7, 5, 3, 3, 5)]
    for _ in range(300):
        n1, n2 = (int(x) for x in rng.integers(2, 400, 2))
        n3 = int(rng.integers(1, 400))
        cases.append((n1, n2, n3, int(rng.integers(1, n3 + 1)), int(rng.integers(1, min(n1, n2) + 1))))
    for (l, m, n, p, k) in cases:
        for v in (0, 1):
            assert b.hosvd_matched_k2(l, m, n, p, k, v) == oracle.hosvd_matched_k2(l, m, n, p, k, v), \
                (l, m, n, p, k, v)
    L = b.lib()
    out = ctypes.c_int64(-1)
    assert L.pp_hosvd_matched_k2(10, 10, 10, 2, 3, 2, ctypes.byref(out)) == b.PP_EINVAL
    assert L.pp_hosvd_matched_k2(10, 10, 10, 2, 3, 0, None) == b.PP_EINVAL
    assert L.pp_hosvd_matched_k2(10, 10, 10, 11, 3, 0, ctypes.byref(out)) == b.PP_ESHAPE
    assert L.pp_hosvd_matched_k2(10, 10, 10, 2, 11, 0, ctypes.byref(out)) == b.PP_ESHAPE


def test_u3_builder_host_validation():
    b = _lib()
    L = b.lib()
    assert b.workspace_bytes(b.PP_OP_U3, l=120, m=160, n=300, p=50) > 300 * 300 * 4
    assert L.pprod_u3(None, 4, 4, 8, 2, FAKE, None, None, None, FAKE, 1 << 30, None) == b.PP_EINVAL
    assert L.pprod_u3(FAKE, 4, 4, 8, 9, FAKE, None, None, None, FAKE, 1 << 30, None) == b.PP_ESHAPE
    assert L.pprod_u3(FAKE, 4, 4, 1000, 9, FAKE, None, None, None, FAKE, 1 << 40, None) == b.PP_ENOSYS
    assert L.pprod_u3(FAKE, 4, 4, 8, 2, FAKE, None, None, None, FAKE, 16, None) == b.PP_EWORKSPACE


def test_complex_entry_points_validate_on_host():
    b = _lib()
    L = b.lib()
    o = b.pp_opts()
    # mismatched A_k pointers, NULL factors, bad k, gamma, slice too large for the complex Jacobi
    assert L.tsvdq_trunc_c(FAKE, FAKE, 4, 6, 8, 2, 2, FAKE, FAKE, FAKE, FAKE, None, None,
                           ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_EINVAL
    assert L.tsvdq_trunc_c(FAKE, FAKE, 4, 6, 8, 2, 2, None, FAKE, FAKE, None, None, None,
                           ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_EINVAL
    assert L.tsvdq_trunc_c(FAKE, FAKE, 4, 6, 8, 2, 5, FAKE, FAKE, FAKE, None, None, None,
                           ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_ESHAPE
    for g in (0.0, 1.5):
        assert L.tsvdqII_c(FAKE, FAKE, 4, 6, 8, 2, g, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                           None, ctypes.byref(o), FAKE, 1 << 30, None) == b.PP_EINVAL
    assert L.tsvdqII_c(FAKE, FAKE, 400, 400, 8, 2, 0.9, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                       None, ctypes.byref(o), FAKE, 1 << 40, None) == b.PP_ENOSYS
    assert L.tsvdqII_c(FAKE, FAKE, 4, 6, 8, 2, 0.9, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                       None, ctypes.byref(o), FAKE, 16, None) == b.PP_EWORKSPACE
    assert L.pprod_c(FAKE, FAKE, FAKE, 3, 3, 3, 4, 5, FAKE, FAKE, FAKE, 1 << 20, None) == b.PP_ESHAPE
    assert b.workspace_bytes(b.PP_OP_TSVDQII_C, l=120, m=160, n=300, p=50) > \
        2 * b.workspace_bytes(b.PP_OP_PPROD_C, l=4, m=4, n=8, p=2, n2=4)
