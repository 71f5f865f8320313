"""Differentiable projected product: the hand-written backward (pprod_backward,
through the autograd Function) against the oracle's FP64 gradient, which is
itself pinned to central finite differences.  Tolerance: relative Frobenius
error <= 1e-5 per gradient (the FP32 path's per-stage error is ~2.5e-7; four
chained products and an n*p reduction over all pixels stay an order below)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    x = x.double().cpu().numpy() if torch.is_tensor(x) else x
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def _qr(n, p, gen):
    Q, _ = torch.linalg.qr(torch.randn((n, p), generator=gen, dtype=torch.float64))
    return Q.contiguous()


def _instance(n, n1, m, n2, p, seed, bf16=False):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((n, n1, m), generator=g, dtype=torch.float64) / np.sqrt(n1)
    B = torch.randn((n, m, n2), generator=g, dtype=torch.float64) / np.sqrt(m)
    Q = _qr(n, p, g)
    As = torch.randn((n, n1, m), generator=g, dtype=torch.float64) / np.sqrt(n1)
    Qs = _qr(n, p, g)
    if bf16:                                  # BF16-valued inputs (config: W, X stored in BF16)
        A, B, As = (x.to(torch.bfloat16).double() for x in (A, B, As))
    A, B, Q, As, Qs = (x.float().contiguous() for x in (A, B, Q, As, Qs))
    T = torch.from_numpy(oracle.qprod(As.numpy(), B.numpy(), Qs.numpy())).float()  # teacher
    return A, B, Q, T


def _check(A, B, Q, T, tol=1e-5):
    from paper_2409_19402_gb300 import autograd as ag
    import __graft_entry__
    __graft_entry__.build()
    Ad, Bd, Qd, Td = (x.cuda().requires_grad_(i < 3) for i, x in enumerate((A, B, Q, T)))
    C = ag.qprod(Ad, Bd, Qd)
    loss = 0.5 * ((C - Td) ** 2).sum()
    loss.backward()
    L0, dA, dB, dQE, dQ = oracle.qprod_grad(A.numpy(), B.numpy(), Q.numpy(), T.numpy())
    assert float(loss.detach()) == pytest.approx(L0, rel=1e-5)
    for got, ref, name in ((Ad.grad, dA, "dA"), (Bd.grad, dB, "dB"), (Qd.grad, dQ, "dQ")):
        assert _rel(got, ref) <= tol, (name, _rel(got, ref))
    return Ad, Bd, Qd


def test_gradients_on_the_finite_difference_instance():
    A, B, Q, T = _instance(32, 16, 12, 10, 8, seed=4)
    Ad, Bd, Qd = _check(A, B, Q, T)
    S = Qd.detach().double().T @ Qd.grad.double()          # tangent: Q^T dQ skew-symmetric
    assert float((S + S.T).abs().max()) <= 1e-5 * float(Qd.grad.abs().max())


def test_euclidean_gradient_and_projection():
    from paper_2409_19402_gb300 import binding
    A, B, Q, T = _instance(48, 20, 18, 14, 12, seed=5)
    Ad, Bd, Qd, Td = (x.cuda() for x in (A, B, Q, T))
    C = binding.pprod(Ad, Bd, Qd)
    dA, dB, dQ, dQE = binding.pprod_backward(Ad, Bd, Qd, (C - Td).contiguous(), want_euclid=True)
    torch.cuda.synchronize()
    _, rA, rB, rQE, rQ = oracle.qprod_grad(A.numpy(), B.numpy(), Q.numpy(), T.numpy())
    assert _rel(dQE, rQE) <= 1e-5 and _rel(dQ, rQ) <= 1e-5
    assert _rel(dA, rA) <= 1e-5 and _rel(dB, rB) <= 1e-5


def test_config_size_bf16_inputs():
    """W 256x256x512, X 256x64x512 (BF16 values), Q 512x64, teacher from (W*, Q*)."""
    A, B, Q, T = _instance(512, 256, 256, 64, 64, seed=4, bf16=True)
    _check(A, B, Q, T)


def test_descent_step_with_retraction():
    from paper_2409_19402_gb300 import autograd as ag
    A, B, Q, T = _instance(64, 24, 20, 16, 16, seed=6)
    Ad, Bd, Qd, Td = (x.cuda() for x in (A, B, Q, T))
    Ad.requires_grad_(); Bd.requires_grad_(); Qd.requires_grad_()
    loss0 = 0.5 * ((ag.qprod(Ad, Bd, Qd) - Td) ** 2).sum()
    loss0.backward()
    lr = 1e-2
    with torch.no_grad():
        A1 = Ad - lr * Ad.grad
        B1 = Bd - lr * Bd.grad
        Q1, R = torch.linalg.qr(Qd - lr * Qd.grad)                 # retraction onto St_{n,p}
        Q1 = (Q1 * torch.sign(torch.diagonal(R))).contiguous()
        loss1 = 0.5 * ((ag.qprod(A1, B1, Q1) - Td) ** 2).sum()
    assert float(loss1) < float(loss0)


@pytest.mark.parametrize("dims", [
    (96, 100, 52, 36, 20),     # faces wider than tall: C_t, dA_t, dB_t stored transposed
    (64, 36, 60, 132, 16),     # faces taller than wide: stored directly
    (48, 8, 2048, 4, 40),      # 40 faces of 1 MB images, 32 to a launch: two launches
])
def test_forward_and_backward_on_the_batched_tile_layouts(dims):
    """The facewise products of pprod and pprod_backward in each operand layout
    of the warp-specialised kernel (contraction- or pixel-contiguous X, direct
    or transposed store), ragged in every tile dimension, against the oracle."""
    from paper_2409_19402_gb300 import binding
    n, n1, m, n2, p = dims
    A, B, Q, T = _instance(n, n1, m, n2, p, seed=11)
    Ad, Bd, Qd, Td = (x.cuda() for x in (A, B, Q, T))
    C = binding.pprod(Ad, Bd, Qd)
    torch.cuda.synchronize()
    assert _rel(C, oracle.qprod(A.numpy(), B.numpy(), Q.numpy())) <= 1e-5
    dA, dB, dQ, dQE = binding.pprod_backward(Ad, Bd, Qd, (C - Td).contiguous(), want_euclid=True)
    torch.cuda.synchronize()
    _, rA, rB, rQE, rQ = oracle.qprod_grad(A.numpy(), B.numpy(), Q.numpy(), T.numpy())
    for got, ref, name in ((dA, rA, "dA"), (dB, rB, "dB"), (dQE, rQE, "dQE"), (dQ, rQ, "dQ")):
        assert _rel(got, ref) <= 1e-5, (name, _rel(got, ref))
