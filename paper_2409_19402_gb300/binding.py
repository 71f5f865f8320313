"""Thin ctypes binding of the C ABI in include/pprod.h (same names).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libpprod.so``.  PyTorch supplies device memory (outputs and the
workspace are allocated here, by the caller side of the ABI) and the current
CUDA stream.  There is no CPU fallback: if the library is missing or a CUDA
device is absent the calls raise.

Tensors follow the library's layout: an l x m x n tensor is a C-contiguous
FP32 CUDA tensor of shape (n, l, m); Q is (n, p).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpprod.so")

PP_OK, PP_EINVAL, PP_ESHAPE, PP_ENOTORTHO, PP_ENONFINITE, PP_ENOCONV = 0, 1, 2, 3, 4, 5
PP_ETIMEOUT, PP_EWORKSPACE, PP_ECUDA, PP_ENOSYS = 6, 7, 8, 9
PP_OP_MODE3, PP_OP_FACEWISE, PP_OP_PPROD, PP_OP_TSVDQ, PP_OP_TSVDQII, PP_OP_HOSVD = 0, 1, 2, 3, 4, 5
PP_OP_PPROD_BWD = 6
PP_OP_U3 = 7
PP_OP_PPROD_C, PP_OP_TSVDQ_C, PP_OP_TSVDQII_C = 8, 9, 10


class PPError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)}")
        self.status = status


class pp_shape(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("l", "m", "n", "p", "k", "n2")]


class pp_opts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("check_q", ctypes.c_int32),
                ("q_tol", ctypes.c_float), ("check_finite", ctypes.c_int32),
                ("jacobi_tol", ctypes.c_float), ("precond", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class pp_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("K", ctypes.c_int64),
                ("kappa", ctypes.c_int64), ("normA2", ctypes.c_double),
                ("normAh2", ctypes.c_double), ("kept2", ctypes.c_double),
                ("discarded2", ctypes.c_double), ("err2", ctypes.c_double),
                ("proj_err2", ctypes.c_double)]


class pp_batch_item(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("l", ctypes.c_int64),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("rho", ctypes.c_void_p), ("offs", ctypes.c_void_p), ("Uh_pk", ctypes.c_void_p),
                ("s_pk", ctypes.c_void_p), ("Vh_pk", ctypes.c_void_p), ("Ak", ctypes.c_void_p),
                ("rep", ctypes.c_void_p), ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t)]


class pp_hosvd_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("k1", ctypes.c_int64),
                ("k2", ctypes.c_int64), ("k", ctypes.c_int64), ("normA2", ctypes.c_double),
                ("err2_hosvd", ctypes.c_double), ("err2_tsvdq", ctypes.c_double),
                ("proj_err2", ctypes.c_double)]


REPORT_BYTES = ctypes.sizeof(pp_report)
HOSVD_REPORT_BYTES = ctypes.sizeof(pp_hosvd_report)
_lib = None


def lib() -> ctypes.CDLL:
    """Load libpprod.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
        L.pp_status_str.argtypes = [i32]
        L.pp_status_str.restype = ctypes.c_char_p
        L.pp_version.restype = ctypes.c_char_p
        L.pp_workspace_bytes.argtypes = [i32, ctypes.POINTER(pp_shape)]
        L.pp_workspace_bytes.restype = sz
        L.pprod_mode3.argtypes = [vp, i64, i64, i64, vp, i64, i32, vp, vp]
        L.pprod_facewise.argtypes = [vp, vp, i64, i64, i64, i64, vp, vp]
        L.pprod.argtypes = [vp, vp, vp, i64, i64, i64, i64, i64, vp, vp, sz, vp]
        L.tsvdq_trunc.argtypes = [vp, vp, i64, i64, i64, i64, i64, vp, vp, vp, vp, vp,
                                  ctypes.POINTER(pp_opts), vp, sz, vp]
        L.tsvdqII.argtypes = [vp, vp, i64, i64, i64, i64, ctypes.c_double, vp, vp, vp, vp, vp,
                              vp, vp, ctypes.POINTER(pp_opts), vp, sz, vp]
        for f in ("pprod_mode3", "pprod_facewise", "pprod", "tsvdq_trunc", "tsvdqII"):
            getattr(L, f).restype = i32
        L.pprod_backward.argtypes = [vp, vp, vp, vp, i64, i64, i64, i64, i64, vp, vp, vp, vp,
                                     vp, sz, vp]
        L.pprod_backward.restype = i32
        L.tsvdqII_batched.argtypes = [ctypes.POINTER(pp_batch_item), i64, ctypes.c_double,
                                      ctypes.POINTER(pp_opts), vp]
        L.tsvdqII_batched.restype = i32
        L.hosvd_compare.argtypes = [vp, vp, i64, i64, i64, i64, i64, i64, vp, vp,
                                    ctypes.POINTER(pp_opts), vp, sz, vp]
        L.hosvd_compare.restype = i32
        L.tsvdqII_noalloc.argtypes = [vp, vp, i64, i64, i64, i64, ctypes.c_double, vp, vp, vp,
                                      vp, vp, vp, vp, ctypes.POINTER(pp_opts), vp]
        L.tsvdqII_noalloc.restype = i32
        L.pprod_c.argtypes = [vp, vp, vp, i64, i64, i64, i64, i64, vp, vp, vp, sz, vp]
        L.tsvdq_trunc_c.argtypes = [vp, vp, i64, i64, i64, i64, i64, vp, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(pp_opts), vp, sz, vp]
        L.tsvdqII_c.argtypes = [vp, vp, i64, i64, i64, i64, ctypes.c_double, vp, vp, vp, vp, vp,
                                vp, vp, vp, ctypes.POINTER(pp_opts), vp, sz, vp]
        for f in ("pprod_c", "tsvdq_trunc_c", "tsvdqII_c"):
            getattr(L, f).restype = i32
        L.pprod_u3.argtypes = [vp, i64, i64, i64, i64, vp, vp, vp, ctypes.POINTER(pp_opts), vp,
                               sz, vp]
        L.pprod_u3.restype = i32
        L.pp_hosvd_matched_k2.argtypes = [i64, i64, i64, i64, i64, i32, ctypes.POINTER(i64)]
        L.pp_hosvd_matched_k2.restype = i32
        L.pp_set_jacobi_shape.argtypes = [i64, i64, i64, i32, i32]
        L.pp_set_jacobi_shape.restype = i32
        L.pp_set_stage_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32]
        L.pp_set_stage_events.restype = None
        L.pp_kernel_launches.restype = ctypes.c_uint64
        L.pp_peak_probe.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double), vp, vp]
        L.pp_peak_probe.restype = i32
        _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().pp_status_str(int(status)).decode()


def version() -> str:
    return lib().pp_version().decode()


def kernel_launches() -> int:
    """Process-wide count of kernels launched by libpprod.so."""
    return int(lib().pp_kernel_launches())


def peak_probe(kind: int, reps: int, stream=None) -> float:
    """Enqueue the arithmetic-peak probe (0: FP32 FMA, 1: tcgen05 tf32) on
    `stream`; returns the flops the launch performs (time it with events)."""
    fl = ctypes.c_double(0.0)
    _raise(lib().pp_peak_probe(int(kind), int(reps), ctypes.byref(fl), None, _stream(stream)),
           "pp_peak_probe")
    return fl.value


def set_stage_events(events) -> None:
    """Register torch.cuda.Event objects (already recorded once, so that they
    exist) as stage-boundary events of tsvdq_trunc / tsvdqII; None clears."""
    if not events:
        lib().pp_set_stage_events(None, 0)
        return
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    lib().pp_set_stage_events(arr, len(events))


def set_jacobi_shape(l: int, m: int, p: int, C: int, GW: int = 16) -> None:
    """Register the Jacobi launch shape for l x m slices, p per call (C = 0 removes it)."""
    _raise(lib().pp_set_jacobi_shape(int(l), int(m), int(p), int(C), int(GW)), "pp_set_jacobi_shape")


def workspace_bytes(op: int, l=0, m=0, n=0, p=0, k=0, n2=0) -> int:
    sh = pp_shape(l, m, n, p, k, n2)
    return int(lib().pp_workspace_bytes(op, ctypes.byref(sh)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check_t(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")


def _raise(st: int, what: str):
    if st != PP_OK:
        raise PPError(st, what)


def _opts(max_sweeps=0, check_q=False, q_tol=0.0, check_finite=False, jacobi_tol=0.0,
          precond=True):
    return pp_opts(int(max_sweeps), int(bool(check_q)), float(q_tol), int(bool(check_finite)),
                   float(jacobi_tol), 0 if precond else -1)


def workspace(nbytes: int, device) -> torch.Tensor | None:
    return None if nbytes == 0 else torch.empty(nbytes, dtype=torch.uint8, device=device)


def read_report(rep: torch.Tensor) -> pp_report:
    """Copy a device pp_report (uint8 tensor) to the host and unpack it."""
    raw = bytes(rep.cpu().numpy().tobytes())
    return pp_report.from_buffer_copy(raw)


# --------------------------------------------------------------- entry points
def pprod_mode3(X: torch.Tensor, Q: torch.Tensor, transpose: int, out=None, stream=None):
    """Def. 2.2: transpose=0 -> X x_3 Q^T (n -> p slices); 1 -> X x_3 Q (p -> n)."""
    _check_t(X, "X"); _check_t(Q, "Q")
    n, p = Q.shape
    s_in, l, m = X.shape
    if s_in != (n if transpose == 0 else p):
        raise ValueError("X slice count does not match Q")
    if out is None:
        out = torch.empty(((p if transpose == 0 else n), l, m), dtype=torch.float32,
                          device=X.device)
    _raise(lib().pprod_mode3(_ptr(X), l, m, n, _ptr(Q), p, int(transpose), _ptr(out),
                             _stream(stream)), "pprod_mode3")
    return out


def pprod_facewise(Ah: torch.Tensor, Bh: torch.Tensor, out=None, stream=None):
    """Def. 2.3: Ch[t] = Ah[t] @ Bh[t]."""
    _check_t(Ah, "Ah"); _check_t(Bh, "Bh")
    p, n1, m = Ah.shape
    n2 = Bh.shape[2]
    if out is None:
        out = torch.empty((p, n1, n2), dtype=torch.float32, device=Ah.device)
    _raise(lib().pprod_facewise(_ptr(Ah), _ptr(Bh), n1, m, n2, p, _ptr(out), _stream(stream)),
           "pprod_facewise")
    return out


def pprod(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, out=None, ws=None, stream=None):
    """Def. 3.1: A *Q B."""
    _check_t(A, "A"); _check_t(B, "B"); _check_t(Q, "Q")
    n, n1, m = A.shape
    n2 = B.shape[2]
    p = Q.shape[1]
    if out is None:
        out = torch.empty((n, n1, n2), dtype=torch.float32, device=A.device)
    need = workspace_bytes(PP_OP_PPROD, l=n1, m=m, n=n, p=p, n2=n2)
    if ws is None:
        ws = workspace(need, A.device)
    _raise(lib().pprod(_ptr(A), _ptr(B), _ptr(Q), n1, m, n2, n, p, _ptr(out), _ptr(ws),
                       0 if ws is None else ws.numel(), _stream(stream)), "pprod")
    return out


def pprod_backward(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, G: torch.Tensor,
                   want_euclid: bool = False, ws=None, stream=None):
    """Backward of A *Q B for dL/dC = G: returns (dA, dB, dQ_stiefel, dQ_euclid or None)."""
    for t, nm in ((A, "A"), (B, "B"), (Q, "Q"), (G, "G")):
        _check_t(t, nm)
    n, n1, m = A.shape
    n2 = B.shape[2]
    p = Q.shape[1]
    dA, dB = torch.empty_like(A), torch.empty_like(B)
    dQ = torch.empty_like(Q)
    dQE = torch.empty_like(Q) if want_euclid else None
    need = workspace_bytes(PP_OP_PPROD_BWD, l=n1, m=m, n=n, p=p, n2=n2)
    if ws is None:
        ws = workspace(need, A.device)
    _raise(lib().pprod_backward(_ptr(A), _ptr(B), _ptr(Q), _ptr(G), n1, m, n2, n, p, _ptr(dA),
                                _ptr(dB), _ptr(dQE), _ptr(dQ), _ptr(ws),
                                0 if ws is None else ws.numel(), _stream(stream)), "pprod_backward")
    return dA, dB, dQ, dQE


@dataclass
class TsvdqOut:
    Uh: torch.Tensor     # (p, l, k)
    s: torch.Tensor      # (p, k)
    Vh: torch.Tensor     # (p, m, k)
    Ak: torch.Tensor | None
    rep: torch.Tensor    # device pp_report bytes

    def report(self) -> pp_report:
        return read_report(self.rep)


def tsvdq_trunc(A: torch.Tensor, Q: torch.Tensor, k: int, want_ak: bool = True, ws=None,
                stream=None, **opts) -> TsvdqOut:
    """Alg. 4.1 truncated *Q-SVD."""
    _check_t(A, "A"); _check_t(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    dev = A.device
    Uh = torch.empty((p, l, k), dtype=torch.float32, device=dev)
    s = torch.empty((p, k), dtype=torch.float32, device=dev)
    Vh = torch.empty((p, m, k), dtype=torch.float32, device=dev)
    Ak = torch.empty((n, l, m), dtype=torch.float32, device=dev) if want_ak else None
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_TSVDQ, l=l, m=m, n=n, p=p, k=k)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().tsvdq_trunc(_ptr(A), _ptr(Q), l, m, n, p, int(k), _ptr(Uh), _ptr(s), _ptr(Vh),
                             _ptr(Ak), _ptr(rep), ctypes.byref(o), _ptr(ws),
                             0 if ws is None else ws.numel(), _stream(stream)), "tsvdq_trunc")
    return TsvdqOut(Uh, s, Vh, Ak, rep)


@dataclass
class TsvdqIIOut:
    rho: torch.Tensor    # (p,) int32
    offs: torch.Tensor   # (p+1,) int64
    Uh: torch.Tensor     # packed, capacity p*r*l
    s: torch.Tensor      # packed, capacity p*r
    Vh: torch.Tensor     # packed, capacity p*r*m
    Ak: torch.Tensor | None
    rep: torch.Tensor
    l: int
    m: int

    def report(self) -> pp_report:
        return read_report(self.rep)

    def slices(self):
        """Per-slice host copies [(Uh_t (l, rho_t), s_t, Vh_t (m, rho_t)), ...]."""
        rho = self.rho.cpu().tolist()
        offs = self.offs.cpu().tolist()
        U, S, V = self.Uh.cpu(), self.s.cpu(), self.Vh.cpu()
        out = []
        for t, r in enumerate(rho):
            o = offs[t]
            out.append((U[self.l * o: self.l * o + self.l * r].reshape(self.l, r),
                        S[o: o + r], V[self.m * o: self.m * o + self.m * r].reshape(self.m, r)))
        return out


def tsvdqII(A: torch.Tensor, Q: torch.Tensor, gamma: float, want_ak: bool = True, ws=None,
            stream=None, **opts) -> TsvdqIIOut:
    """Alg. 4.2 *Q-SVDII."""
    _check_t(A, "A"); _check_t(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    r = min(l, m)
    dev = A.device
    rho = torch.empty(p, dtype=torch.int32, device=dev)
    offs = torch.empty(p + 1, dtype=torch.int64, device=dev)
    Uh = torch.empty(p * r * l, dtype=torch.float32, device=dev)
    s = torch.empty(p * r, dtype=torch.float32, device=dev)
    Vh = torch.empty(p * r * m, dtype=torch.float32, device=dev)
    Ak = torch.empty((n, l, m), dtype=torch.float32, device=dev) if want_ak else None
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_TSVDQII, l=l, m=m, n=n, p=p)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().tsvdqII(_ptr(A), _ptr(Q), l, m, n, p, float(gamma), _ptr(rho), _ptr(offs),
                         _ptr(Uh), _ptr(s), _ptr(Vh), _ptr(Ak), _ptr(rep), ctypes.byref(o),
                         _ptr(ws), 0 if ws is None else ws.numel(), _stream(stream)), "tsvdqII")
    return TsvdqIIOut(rho, offs, Uh, s, Vh, Ak, rep, l, m)


def tsvdqII_noalloc(A: torch.Tensor, Q: torch.Tensor, gamma: float, want_ak: bool = True,
                    stream=None, **opts) -> TsvdqIIOut:
    """Alg. 4.2 through tsvdqII_noalloc: no workspace argument, the library's
    fixed device scratch array is used instead (outputs are still the caller's)."""
    _check_t(A, "A"); _check_t(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    r = min(l, m)
    dev = A.device
    rho = torch.empty(p, dtype=torch.int32, device=dev)
    offs = torch.empty(p + 1, dtype=torch.int64, device=dev)
    Uh = torch.empty(p * r * l, dtype=torch.float32, device=dev)
    s = torch.empty(p * r, dtype=torch.float32, device=dev)
    Vh = torch.empty(p * r * m, dtype=torch.float32, device=dev)
    Ak = torch.empty((n, l, m), dtype=torch.float32, device=dev) if want_ak else None
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    o = _opts(**opts)
    _raise(lib().tsvdqII_noalloc(_ptr(A), _ptr(Q), l, m, n, p, float(gamma), _ptr(rho),
                                 _ptr(offs), _ptr(Uh), _ptr(s), _ptr(Vh), _ptr(Ak), _ptr(rep),
                                 ctypes.byref(o), _stream(stream)), "tsvdqII_noalloc")
    return TsvdqIIOut(rho, offs, Uh, s, Vh, Ak, rep, l, m)


def hosvd_compare(A: torch.Tensor, Q: torch.Tensor, k1: int, k2: int, want_ak: bool = False,
                  ws=None, stream=None, **opts):
    """Sec. 4.2: truncated HOSVD (k1, k2, p) with U3 = Q against the *Q-SVD with
    k = min(k1, k2).  Returns (pp_hosvd_report, A_hosvd or None); synchronises."""
    _check_t(A, "A"); _check_t(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    dev = A.device
    Ak = torch.empty((n, l, m), dtype=torch.float32, device=dev) if want_ak else None
    rep = torch.zeros(HOSVD_REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_HOSVD, l=l, m=m, n=n, p=p, k=k1, n2=k2)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().hosvd_compare(_ptr(A), _ptr(Q), l, m, n, p, int(k1), int(k2), _ptr(Ak),
                               _ptr(rep), ctypes.byref(o), _ptr(ws),
                               0 if ws is None else ws.numel(), _stream(stream)), "hosvd_compare")
    raw = bytes(rep.cpu().numpy().tobytes())
    return pp_hosvd_report.from_buffer_copy(raw), Ak


def _check_c(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor")


def pprod_c(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, ws=None, stream=None):
    """Def. 3.1 with a complex Q (n, p) complex64 and real A (n, n1, m), B (n, m, n2);
    returns (C_re, C_im), each (n, n1, n2)."""
    _check_t(A, "A"); _check_t(B, "B"); _check_c(Q, "Q")
    n, n1, m = A.shape
    n2 = B.shape[2]
    p = Q.shape[1]
    dev = A.device
    Cr = torch.empty((n, n1, n2), dtype=torch.float32, device=dev)
    Ci = torch.empty((n, n1, n2), dtype=torch.float32, device=dev)
    need = workspace_bytes(PP_OP_PPROD_C, l=n1, m=m, n=n, p=p, n2=n2)
    if ws is None:
        ws = workspace(need, dev)
    _raise(lib().pprod_c(_ptr(A), _ptr(B), _ptr(Q), n1, m, n2, n, p, _ptr(Cr), _ptr(Ci), _ptr(ws),
                         0 if ws is None else ws.numel(), _stream(stream)), "pprod_c")
    return Cr, Ci


def tsvdq_trunc_c(A: torch.Tensor, Q: torch.Tensor, k: int, want_ak: bool = True, ws=None,
                  stream=None, **opts) -> TsvdqOut:
    """Alg. 4.1 with a complex Q: Uh, Vh complex64; Ak = (Ak_re, Ak_im) or None."""
    _check_t(A, "A"); _check_c(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    dev = A.device
    Uh = torch.empty((p, l, k), dtype=torch.complex64, device=dev)
    s = torch.empty((p, k), dtype=torch.float32, device=dev)
    Vh = torch.empty((p, m, k), dtype=torch.complex64, device=dev)
    Ak = ((torch.empty((n, l, m), dtype=torch.float32, device=dev),
           torch.empty((n, l, m), dtype=torch.float32, device=dev)) if want_ak else (None, None))
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_TSVDQ_C, l=l, m=m, n=n, p=p, k=k)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().tsvdq_trunc_c(_ptr(A), _ptr(Q), l, m, n, p, int(k), _ptr(Uh), _ptr(s), _ptr(Vh),
                               _ptr(Ak[0]), _ptr(Ak[1]), _ptr(rep), ctypes.byref(o), _ptr(ws),
                               0 if ws is None else ws.numel(), _stream(stream)), "tsvdq_trunc_c")
    return TsvdqOut(Uh, s, Vh, Ak if want_ak else None, rep)


def tsvdqII_c(A: torch.Tensor, Q: torch.Tensor, gamma: float, want_ak: bool = True, ws=None,
              stream=None, **opts) -> TsvdqIIOut:
    """Alg. 4.2 with a complex Q: packed Uh, Vh complex64; Ak = (Ak_re, Ak_im) or None."""
    _check_t(A, "A"); _check_c(Q, "Q")
    n, l, m = A.shape
    p = Q.shape[1]
    r = min(l, m)
    dev = A.device
    rho = torch.empty(p, dtype=torch.int32, device=dev)
    offs = torch.empty(p + 1, dtype=torch.int64, device=dev)
    Uh = torch.empty(p * r * l, dtype=torch.complex64, device=dev)
    s = torch.empty(p * r, dtype=torch.float32, device=dev)
    Vh = torch.empty(p * r * m, dtype=torch.complex64, device=dev)
    Ak = ((torch.empty((n, l, m), dtype=torch.float32, device=dev),
           torch.empty((n, l, m), dtype=torch.float32, device=dev)) if want_ak else (None, None))
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_TSVDQII_C, l=l, m=m, n=n, p=p)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().tsvdqII_c(_ptr(A), _ptr(Q), l, m, n, p, float(gamma), _ptr(rho), _ptr(offs),
                           _ptr(Uh), _ptr(s), _ptr(Vh), _ptr(Ak[0]), _ptr(Ak[1]), _ptr(rep),
                           ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(),
                           _stream(stream)), "tsvdqII_c")
    return TsvdqIIOut(rho, offs, Uh, s, Vh, Ak if want_ak else None, rep, l, m)


def pprod_u3(A: torch.Tensor, p: int, ws=None, stream=None, **opts):
    """U3 transformation (Thm. 4.3): Q (n, p) = leading eigenvectors of A_(3) A_(3)^T,
    lambda (p) their eigenvalues, and the device pp_report (uint8 tensor; read_report)."""
    _check_t(A, "A")
    n, l, m = A.shape
    dev = A.device
    Q = torch.empty((n, p), dtype=torch.float32, device=dev)
    lam = torch.empty((p,), dtype=torch.float32, device=dev)
    rep = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev)
    need = workspace_bytes(PP_OP_U3, l=l, m=m, n=n, p=p)
    if ws is None:
        ws = workspace(need, dev)
    o = _opts(**opts)
    _raise(lib().pprod_u3(_ptr(A), l, m, n, int(p), _ptr(Q), _ptr(lam), _ptr(rep),
                          ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(),
                          _stream(stream)), "pprod_u3")
    return Q, lam, rep


def hosvd_matched_k2(l: int, m: int, n: int, p: int, k: int, variant: int) -> int:
    """Sec. 5.3 storage matching: largest HOSVD rank k2 with multirank (l, k2, p)
    (variant 0) or (k2, k2, p) (variant 1) storing no more than the *Q-SVD with
    truncation k; 0 when none fits.  Host-only."""
    out = ctypes.c_int64(0)
    _raise(lib().pp_hosvd_matched_k2(int(l), int(m), int(n), int(p), int(k), int(variant),
                                     ctypes.byref(out)), "pp_hosvd_matched_k2")
    return int(out.value)


class Batch:
    """Preallocated outputs and workspaces for tsvdqII_batched over a list of
    (A, Q) device tensors; call() enqueues the whole batch on `stream` (no
    allocation, so it can be captured into a CUDA graph and replayed)."""

    def __init__(self, pairs, gamma: float, want_ak: bool = False, **opts):
        self.gamma = float(gamma)
        self.opts = _opts(**opts)
        self.outs = []
        sizes = []
        for A, Q in pairs:
            _check_t(A, "A"); _check_t(Q, "Q")
            n, l, m = A.shape
            sizes.append(workspace_bytes(PP_OP_TSVDQII, l=l, m=m, n=n, p=Q.shape[1]))
        offsets, tot = [], 0
        for nb in sizes:
            offsets.append(tot)
            tot += (nb + 1023) // 1024 * 1024
        dev = pairs[0][0].device
        self.ws = torch.empty(max(tot, 1), dtype=torch.uint8, device=dev)
        items = []
        for (A, Q), off, nb in zip(pairs, offsets, sizes):
            n, l, m = A.shape
            p = Q.shape[1]
            r = min(l, m)
            o = TsvdqIIOut(torch.empty(p, dtype=torch.int32, device=dev),
                           torch.empty(p + 1, dtype=torch.int64, device=dev),
                           torch.empty(p * r * l, dtype=torch.float32, device=dev),
                           torch.empty(p * r, dtype=torch.float32, device=dev),
                           torch.empty(p * r * m, dtype=torch.float32, device=dev),
                           torch.empty((n, l, m), dtype=torch.float32, device=dev) if want_ak else None,
                           torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=dev), l, m)
            self.outs.append(o)
            items.append(pp_batch_item(A.data_ptr(), Q.data_ptr(), l, m, n, p, o.rho.data_ptr(),
                                       o.offs.data_ptr(), o.Uh.data_ptr(), o.s.data_ptr(),
                                       o.Vh.data_ptr(), 0 if o.Ak is None else o.Ak.data_ptr(),
                                       o.rep.data_ptr(), self.ws.data_ptr() + off, nb))
        self.pairs = pairs
        self.items = (pp_batch_item * len(items))(*items)

    def __call__(self, stream=None):
        _raise(lib().tsvdqII_batched(self.items, len(self.outs), self.gamma,
                                     ctypes.byref(self.opts), _stream(stream)), "tsvdqII_batched")
        return self.outs
