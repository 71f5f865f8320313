"""Batched uneven workload (64 tensors, l, m ~ U{32..256}, n ~ U{64..512},
p ~ U{8..64}, Tucker rank 10 + noise; Q = U3 per tensor; gamma = 0.95):
tsvdqII_batched must give, tensor by tensor, bit-identical results to the
single-tensor tsvdqII (same kernels and launch shapes), the single calls of
the smallest tensors are checked against the oracle with the parity
tolerances, and a CUDA-graph capture of the batch must replay to the same
results."""
import numpy as np
import pytest
import torch

from paper_2409_19402_gb300 import inputs
from tests.test_gpu_parity import _tsvdqII_case

pytestmark = pytest.mark.gpu
GAMMA = 0.95


@pytest.fixture(scope="module")
def batch():
    items = inputs.batched()
    return [(A, inputs.u3_q(A, p)) for A, p in items]


def _b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_19402_gb300 import binding
    return binding


def _dev(batch):
    return [(torch.from_numpy(A).cuda(), torch.from_numpy(Q).cuda()) for A, Q in batch]


def _same(o1, o2):
    assert torch.equal(o1.rho, o2.rho) and torch.equal(o1.offs, o2.offs)
    k = int(o1.offs[-1])
    assert torch.equal(o1.s[:k], o2.s[:k])
    assert torch.equal(o1.Uh[:k * o1.l], o2.Uh[:k * o2.l])
    assert torch.equal(o1.Vh[:k * o1.m], o2.Vh[:k * o2.m])
    assert bytes(o1.rep.cpu().numpy()) == bytes(o2.rep.cpu().numpy())


def test_batched_equals_single_calls(batch):
    b = _b()
    pairs = _dev(batch)
    B = b.Batch(pairs, GAMMA)
    outs = B()
    torch.cuda.synchronize()
    for (A, Q), o in zip(pairs, outs):
        rep = o.report()
        assert rep.status == 0, b.status_str(rep.status)
        single = b.tsvdqII(A, Q, GAMMA, want_ak=False)
        torch.cuda.synchronize()
        _same(o, single)


def test_batched_smallest_against_oracle(batch):
    order = sorted(range(len(batch)), key=lambda i: batch[i][0].size)
    for i in order[:3]:
        A, Q = batch[i]
        _tsvdqII_case(A, Q, GAMMA)


def test_batched_cuda_graph_replay(batch):
    b = _b()
    pairs = _dev(batch[:16])
    B = b.Batch(pairs, GAMMA)
    eager = [(o.rho.clone(), o.offs.clone(), o.s.clone(), o.rep.clone()) for o in B()]
    torch.cuda.synchronize()
    for o in B.outs:
        o.s.zero_()
        o.rep.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for (rho, offs, sv, rep), o in zip(eager, B.outs):
        assert torch.equal(rho, o.rho) and torch.equal(offs, o.offs)
        k = int(offs[-1])                       # entries past kappa are never written
        assert torch.equal(sv[:k], o.s[:k])
        assert torch.equal(rep, o.rep)


def test_batched_every_tensor_sampled_slices_and_ranks(batch):
    """Every tensor of the batch, at any size: the singular values of its first
    and last transform-domain slice recomputed one by one by the oracle, each
    slice's error within 1e-5 of the norm of all the tensor's singular values
    (the normwise parity tolerance, of which a slice's share is a necessary
    part; the last slices of these rank-10 tensors hold noise-level values,
    whose own norm is far below the rounding of the FP32 projection), and the
    batch's ranks rho equal to the global energy selection (Alg. 4.2 steps
    4-7, the oracle's) applied to the same kernels' full singular values, bit
    for bit."""
    import concurrent.futures as cf
    import os

    import oracle
    b = _b()
    pairs = _dev(batch)
    B = b.Batch(pairs, GAMMA)
    outs = B()
    torch.cuda.synchronize()
    jobs = []
    for i, ((A, Q), (Ad, Qd), o) in enumerate(zip(batch, pairs, outs)):
        assert o.report().status == 0
        bmin = min(A.shape[1], A.shape[2])
        full = b.tsvdq_trunc(Ad, Qd, bmin, want_ak=False)
        torch.cuda.synchronize()
        sig = full.s.double().cpu().numpy()
        K, rho, _, _ = oracle.select_energy(sig, GAMMA)
        assert np.array_equal(o.rho.cpu().numpy(), rho), i
        assert int(o.offs[-1]) == K, i
        p = Q.shape[1]
        for t in sorted({0, p - 1}):
            jobs.append((i, t, A, Q, sig[t], np.linalg.norm(sig)))

    def one(job):
        i, t, A, Q, s_gpu, norm_all = job
        Ah_t = oracle.mode3(A, np.asarray(Q, np.float64)[:, t:t + 1].T)[0]
        s = oracle.svd(Ah_t)[1]
        return i, t, np.linalg.norm(s_gpu - s) / max(norm_all, 1e-300)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for i, t, err in ex.map(one, jobs):
            assert err <= 1e-5, (i, t, err)
