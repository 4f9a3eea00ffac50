"""PyTorch-facing calls: device tensors in, device tensors out, every step in
the CUDA library. PyTorch supplies device memory, the current stream and the
autograd plumbing.

Bit matrices are int64 CUDA tensors of shape (rows, ld) holding the uint64
words of the C ABI (LSB-first; see `inputs.pack_bits`); `ld` is even.
theta is a float32 CUDA tensor of length m (other float dtypes are cast to
float32 for the kernels; gradients come back in theta's dtype).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import FP32, SPLIT_BF16, SPARSE_FP32, OP_EXPVAL, OP_EXPVAL_GRAD, OP_MMD_LOSS, OP_MMD_LOSS_GRAD, OP_BITFLIP, check

_PRECISIONS = {"fp32": FP32, "split_bf16": SPLIT_BF16, "sparse_fp32": SPARSE_FP32, FP32: FP32,
               SPLIT_BF16: SPLIT_BF16, SPARSE_FP32: SPARSE_FP32}


def precision_code(precision) -> int:
    try:
        return _PRECISIONS[precision]
    except KeyError:
        raise ValueError(f"precision must be 'fp32', 'split_bf16' or 'sparse_fp32', got {precision!r}") from None


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _bits(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.int64 and t.dim() == 2 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous 2-D int64 CUDA tensor of packed words")
    if t.shape[1] % 2:
        raise ValueError(f"{name}: words per row must be even")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _Workspace:
    """Grow-only scratch per (device, stream); calls on one stream are ordered."""

    def __init__(self):
        self._bufs = {}

    def get(self, nbytes: int, device) -> torch.Tensor:
        key = (torch.device(device).index, _stream(device))
        buf = self._bufs.get(key)
        if buf is None or buf.numel() < nbytes:
            buf = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=device)
            self._bufs[key] = buf
        return buf


_WS = _Workspace()


def workspace_bytes(op: int, n: int, m: int, l: int, s: int, N: int = 0, precision="split_bf16") -> int:
    return int(_lib.load().iqp_workspace_bytes(op, n, m, l, s, N, precision_code(precision)))


def parity(n: int, R: torch.Tensor, G: torch.Tensor, ldp: int | None = None) -> torch.Tensor:
    """P[r, j] = (R_r . g_j) mod 2, bit-packed (rows x ldp int64 words)."""
    _bits(R, "R"), _bits(G, "G")
    m = G.shape[0]
    if ldp is None:
        ldp = (m + 63) // 64
        ldp += ldp & 1
    P = torch.empty((R.shape[0], ldp), dtype=torch.int64, device=R.device)
    check(_lib.load().iqp_parity(n, _ptr(R), R.shape[0], R.shape[1], _ptr(G), m, G.shape[1], _ptr(P), ldp,
                                 ctypes.c_void_p(_stream(R.device))), "iqp_parity")
    return P


def parity_gather(n: int, R: torch.Tensor, G: torch.Tensor):
    """(P, P^T) by the support-gather method: P is rows x ldp words (bits over
    gates), P^T is m x ldpt words (bits over rows)."""
    _bits(R, "R"), _bits(G, "G")
    rows, m = R.shape[0], G.shape[0]
    ldp = (m + 63) // 64
    ldp += ldp & 1
    ldpt = (rows + 63) // 64
    ldpt += ldpt & 1
    P = torch.empty((rows, ldp), dtype=torch.int64, device=R.device)
    PT = torch.empty((m, ldpt), dtype=torch.int64, device=R.device)
    scratch = torch.empty((n, ldpt), dtype=torch.int64, device=R.device)
    check(_lib.load().iqp_parity_gather(n, _ptr(R), rows, R.shape[1], _ptr(G), m, G.shape[1], _ptr(P), ldp, _ptr(PT),
                                        ldpt, _ptr(scratch), ctypes.c_void_p(_stream(R.device))), "iqp_parity_gather")
    return P, PT


def parity_sum(n: int, A: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """T[a] = sum_x (-1)^{a.x} (int64)."""
    _bits(A, "A"), _bits(X, "X")
    T = torch.empty(A.shape[0], dtype=torch.int64, device=A.device)
    check(_lib.load().iqp_parity_sum(n, _ptr(A), A.shape[0], A.shape[1], _ptr(X), X.shape[0], X.shape[1], _ptr(T),
                                     ctypes.c_void_p(_stream(A.device))), "iqp_parity_sum")
    return T


def _theta32(theta: torch.Tensor) -> torch.Tensor:
    if not theta.is_cuda:
        raise ValueError("theta must be a CUDA tensor")
    return theta.detach().to(torch.float32).contiguous()


def expval_raw(n, theta, G, A, Z, precision="split_bf16"):
    """(expval, std_err) as float64 tensors, no autograd."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    prec = precision_code(precision)
    lib = _lib.load()
    nbytes = lib.iqp_workspace_bytes(OP_EXPVAL, n, m, l, s, 0, prec)
    ws = _WS.get(nbytes, G.device)
    ev = torch.empty(l, dtype=torch.float64, device=G.device)
    se = torch.empty(l, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(th), prec,
                         _ptr(ev), _ptr(se), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(G.device))), "iqp_expval")
    return ev, se


def expval_grad(n, theta, G, A, Z, alpha, beta=None, precision="split_bf16") -> torch.Tensor:
    """grad[j] = sum_a sum_i sin Phi (alpha_a + beta_a cos Phi) dPhi/dtheta_j (float64)."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    prec = precision_code(precision)
    al = alpha.detach().to(device=G.device, dtype=torch.float64).contiguous()
    be = None if beta is None else beta.detach().to(device=G.device, dtype=torch.float64).contiguous()
    lib = _lib.load()
    nbytes = lib.iqp_workspace_bytes(OP_EXPVAL_GRAD, n, m, l, s, 0, prec)
    ws = _WS.get(nbytes, G.device)
    grad = torch.empty(m, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval_grad(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(th),
                              _ptr(al), _ptr(be), prec, _ptr(grad), _ptr(ws), ws.numel(),
                              ctypes.c_void_p(_stream(G.device))), "iqp_expval_grad")
    return grad


class _ExpvalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, Z, n, precision):
        ev, se = expval_raw(n, theta, G, A, Z, precision)
        ctx.save_for_backward(theta, G, A, Z)
        ctx.n, ctx.precision = n, precision
        ctx.mark_non_differentiable(se)
        return ev, se

    @staticmethod
    def backward(ctx, g_ev, g_se):
        theta, G, A, Z = ctx.saved_tensors
        if g_ev is None:
            return (None,) * 6
        s = Z.shape[0]
        alpha = -g_ev.to(torch.float64) / s
        grad = expval_grad(ctx.n, theta, G, A, Z, alpha, None, ctx.precision)
        return grad.to(theta.dtype), None, None, None, None, None


def expval(theta, G, A, Z, n: int, precision="split_bf16"):
    """Monte-Carlo <Z_a> estimates and standard errors (float64), differentiable
    in theta (std_err is not)."""
    return _ExpvalFn.apply(theta, G, A, Z, n, precision)


def mmd_loss_raw(n, theta, G, A, Z, X, precision="split_bf16", unbiased=True, with_grad=False):
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z"), (X, "X")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s, N = G.shape[0], A.shape[0], Z.shape[0], X.shape[0]
    prec = precision_code(precision)
    lib = _lib.load()
    op = OP_MMD_LOSS_GRAD if with_grad else OP_MMD_LOSS
    ws = _WS.get(lib.iqp_workspace_bytes(op, n, m, l, s, N, prec), G.device)
    loss = torch.empty(1, dtype=torch.float64, device=G.device)
    st = ctypes.c_void_p(_stream(G.device))
    args = (n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(X), N, X.shape[1],
            _ptr(th), prec, 1 if unbiased else 0)
    if with_grad:
        grad = torch.empty(m, dtype=torch.float64, device=G.device)
        check(lib.iqp_mmd_loss_grad(*args, _ptr(loss), _ptr(grad), _ptr(ws), ws.numel(), st), "iqp_mmd_loss_grad")
        return loss[0], grad
    check(lib.iqp_mmd_loss(*args, _ptr(loss), _ptr(ws), ws.numel(), st), "iqp_mmd_loss")
    return loss[0], None


class _MmdFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, Z, X, n, precision, unbiased):
        loss, grad = mmd_loss_raw(n, theta, G, A, Z, X, precision, unbiased, with_grad=theta.requires_grad)
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=theta.device))
        ctx.theta_dtype = theta.dtype
        return loss

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g.to(torch.float64) * grad).to(ctx.theta_dtype), None, None, None, None, None, None, None


def mmd_loss(theta, G, A, Z, X, n: int, precision="split_bf16", unbiased=True):
    """MMD^2 estimate (float64 scalar tensor), differentiable in theta: the loss
    and its gradient come from one library call (the backward recomputes Phi
    tile by tile inside it)."""
    return _MmdFn.apply(theta, G, A, Z, X, n, precision, unbiased)


def bitflip_expval_raw(n, theta, G, A):
    """Exact <Z_a> of the stochastic bitflip circuit (float64), no autograd."""
    _bits(G, "G"), _bits(A, "A")
    th = _theta32(theta)
    m, l = G.shape[0], A.shape[0]
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_BITFLIP, n, m, l, 1, 0, FP32), G.device)
    ev = torch.empty(l, dtype=torch.float64, device=G.device)
    check(lib.iqp_bitflip_expval(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(th), _ptr(ev), _ptr(ws),
                                 ws.numel(), ctypes.c_void_p(_stream(G.device))), "iqp_bitflip_expval")
    return ev


def bitflip_grad(n, theta, G, A, w) -> torch.Tensor:
    """d/dtheta of sum_a w_a <Z_a> for the bitflip circuit (float64)."""
    _bits(G, "G"), _bits(A, "A")
    th = _theta32(theta)
    m, l = G.shape[0], A.shape[0]
    wd = w.detach().to(device=G.device, dtype=torch.float64).contiguous()
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_BITFLIP, n, m, l, 1, 0, FP32), G.device)
    grad = torch.empty(m, dtype=torch.float64, device=G.device)
    check(lib.iqp_bitflip_grad(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(th), _ptr(wd), _ptr(grad),
                               _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(G.device))), "iqp_bitflip_grad")
    return grad


class _BitflipFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, n):
        ev = bitflip_expval_raw(n, theta, G, A)
        ctx.save_for_backward(theta, G, A)
        ctx.n = n
        return ev

    @staticmethod
    def backward(ctx, g):
        theta, G, A = ctx.saved_tensors
        return bitflip_grad(ctx.n, theta, G, A, g).to(theta.dtype), None, None, None


def bitflip_expval(theta, G, A, n: int):
    """Exact expectation values of the stochastic bitflip circuit (Sec. 2.5),
    differentiable in theta."""
    return _BitflipFn.apply(theta, G, A, n)


def read_status(device=None) -> int:
    """Device-side status recorded in the current stream's workspace (clears it)."""
    device = torch.device("cuda") if device is None else torch.device(device)
    ws = _WS.get(256, device)
    return int(_lib.load().iqp_read_status(_ptr(ws), ws.numel(), ctypes.c_void_p(_stream(device))))


def launch_count() -> int:
    return int(_lib.load().iqp_launch_count())


def tensor_path_available() -> bool:
    return bool(_lib.load().iqp_tensor_path_available())


def to_device_bits(words, device="cuda") -> torch.Tensor:
    """numpy uint64 words -> int64 CUDA tensor (same bits)."""
    import numpy as np
    a = np.ascontiguousarray(words, dtype=np.uint64).view(np.int64)
    return torch.from_numpy(a).to(device)
