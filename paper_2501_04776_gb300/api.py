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
from ._lib import FP32, SPLIT_BF16, SPARSE_FP32, LOWORDER_FP32, OP_EXPVAL, OP_EXPVAL_GRAD, OP_MMD_LOSS, OP_MMD_LOSS_GRAD, OP_BITFLIP, check
from ._lib import OP_EXPVAL_INDEP, OP_EXPVAL_INDEP_GRAD, OP_MMD_LOSS_INDEP, OP_MMD_LOSS_GRAD_INDEP
from ._lib import MMD_UNBIASED, MMD_SQRT, MMD_INDEP

_PRECISIONS = {"fp32": FP32, "split_bf16": SPLIT_BF16, "sparse_fp32": SPARSE_FP32, "loworder_fp32": LOWORDER_FP32,
               FP32: FP32, SPLIT_BF16: SPLIT_BF16, SPARSE_FP32: SPARSE_FP32, LOWORDER_FP32: LOWORDER_FP32}


def precision_code(precision) -> int:
    try:
        return _PRECISIONS[precision]
    except KeyError:
        raise ValueError("precision must be 'fp32', 'split_bf16', 'sparse_fp32' or 'loworder_fp32', "
                         f"got {precision!r}") from None


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _bits(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.int64 and t.dim() == 2 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous 2-D int64 CUDA tensor of packed words")
    if t.shape[1] % 2:
        raise ValueError(f"{name}: words per row must be even")
    return t


def _resolve(device) -> torch.device:
    """torch.device with an explicit index ("cuda" -> the current device)."""
    d = torch.device(device)
    if d.type == "cuda" and d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return d


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _Workspace:
    """Grow-only scratch per (device, stream); calls on one stream are ordered."""

    def __init__(self):
        self._bufs = {}

    def get(self, nbytes: int, device) -> torch.Tensor:
        device = _resolve(device)
        key = (device.index, _stream(device))
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
    scratch = torch.empty((n * ldpt + 2 * m,), dtype=torch.int64, device=R.device)  # R^T, then the support list
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


def expval_value_and_grad(n, theta, G, A, Z, alpha, beta=None, precision="split_bf16"):
    """(expval, std_err, grad) from one call, for gradient coefficients known
    before the estimates (for L = sum_a w_a <Z_a>: alpha = -w / s). In
    split BF16 one pass of the phase contraction yields both the statistics
    and the gradient's W (no recompute)."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    prec = precision_code(precision)
    al = alpha.detach().to(device=G.device, dtype=torch.float64).contiguous()
    be = None if beta is None else beta.detach().to(device=G.device, dtype=torch.float64).contiguous()
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_EXPVAL_GRAD, n, m, l, s, 0, prec), G.device)
    ev = torch.empty(l, dtype=torch.float64, device=G.device)
    se = torch.empty(l, dtype=torch.float64, device=G.device)
    grad = torch.empty(m, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval_value_and_grad(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1],
                                        _ptr(th), _ptr(al), _ptr(be), prec, _ptr(ev), _ptr(se), _ptr(grad), _ptr(ws),
                                        ws.numel(), ctypes.c_void_p(_stream(G.device))), "iqp_expval_value_and_grad")
    return ev, se, grad


# Precisions whose statistics pass can keep Phi for the gradient pass.
KEEP_PHI = (SPLIT_BF16, SPARSE_FP32, LOWORDER_FP32)


def phi_ld(s: int) -> int:
    """Smallest row stride (float32 elements) of a kept Phi for s samples."""
    return (s + 63) // 64 * 64


def expval_keep_phi_raw(n, theta, G, A, Z, precision="split_bf16", ld=None):
    """(expval, std_err, phi): iqp_expval that also keeps Phi (l x ld float32,
    ld = phi_ld(s) by default, in the precision's own sample order) for
    expval_grad_from_phi. No autograd."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    prec = precision_code(precision)
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_EXPVAL, n, m, l, s, 0, prec), G.device)
    ev = torch.empty(l, dtype=torch.float64, device=G.device)
    se = torch.empty(l, dtype=torch.float64, device=G.device)
    ld = phi_ld(s) if ld is None else int(ld)
    phi = torch.empty((l, ld), dtype=torch.float32, device=G.device)
    check(lib.iqp_expval_keep_phi(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(th),
                                  prec, _ptr(ev), _ptr(se), _ptr(phi), ld, _ptr(ws), ws.numel(),
                                  ctypes.c_void_p(_stream(G.device))), "iqp_expval_keep_phi")
    return ev, se, phi


def expval_grad_from_phi(n, theta, G, A, Z, phi, alpha, beta=None, precision="split_bf16") -> torch.Tensor:
    """expval_grad with W formed from a Phi that expval_keep_phi_raw kept for
    the same inputs and precision (no second phase pass; same result)."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    prec = precision_code(precision)
    if not (phi.is_cuda and phi.dtype == torch.float32 and phi.dim() == 2 and phi.is_contiguous()
            and phi.shape[0] == l):
        raise ValueError("phi must be the contiguous l x ld float32 CUDA tensor expval_keep_phi_raw returned")
    al = alpha.detach().to(device=G.device, dtype=torch.float64).contiguous()
    be = None if beta is None else beta.detach().to(device=G.device, dtype=torch.float64).contiguous()
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_EXPVAL_GRAD, n, m, l, s, 0, prec), G.device)
    grad = torch.empty(m, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval_grad_from_phi(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1],
                                       _ptr(th), _ptr(al), _ptr(be), prec, _ptr(phi), phi.shape[1], _ptr(grad),
                                       _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(G.device))),
          "iqp_expval_grad_from_phi")
    return grad


class _ExpvalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, Z, n, precision, keep_phi):
        phi = None
        if keep_phi and ctx.needs_input_grad[0] and precision_code(precision) in KEEP_PHI:
            ev, se, phi = expval_keep_phi_raw(n, theta, G, A, Z, precision)
        else:
            ev, se = expval_raw(n, theta, G, A, Z, precision)
        ctx.save_for_backward(theta, G, A, Z, phi)
        ctx.n, ctx.precision = n, precision
        ctx.mark_non_differentiable(se)
        return ev, se

    @staticmethod
    def backward(ctx, g_ev, g_se):
        theta, G, A, Z, phi = ctx.saved_tensors
        if g_ev is None:
            return (None,) * 7
        s = Z.shape[0]
        alpha = -g_ev.to(torch.float64) / s
        if phi is not None:
            grad = expval_grad_from_phi(ctx.n, theta, G, A, Z, phi, alpha, None, ctx.precision)
        else:
            grad = expval_grad(ctx.n, theta, G, A, Z, alpha, None, ctx.precision)
        return grad.to(theta.dtype), None, None, None, None, None, None


def expval(theta, G, A, Z, n: int, precision="split_bf16", keep_phi=True):
    """Monte-Carlo <Z_a> estimates and standard errors (float64), differentiable
    in theta (std_err is not). With keep_phi (split BF16, row-sparse and
    low-order forms) the forward keeps Phi (4 l s bytes, held until the
    backward) so the backward forms W from it instead of recomputing Phi;
    keep_phi=False holds only the inputs and recomputes."""
    return _ExpvalFn.apply(theta, G, A, Z, n, precision, keep_phi)


def mmd_loss_raw(n, theta, G, A, Z, X, precision="split_bf16", unbiased=True, with_grad=False, sqrt_loss=False,
                 indep=False):
    """MMD^2 (or its square root with sqrt_loss) and optionally its gradient.
    indep: observable a uses its own samples, rows a*s..a*s+s-1 of Z."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z"), (X, "X")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l, N = G.shape[0], A.shape[0], X.shape[0]
    if indep and Z.shape[0] % l:
        raise ValueError("indep: Z must have l * s rows")
    s = Z.shape[0] // l if indep else Z.shape[0]
    prec = precision_code(precision)
    lib = _lib.load()
    if indep:
        op = OP_MMD_LOSS_GRAD_INDEP if with_grad else OP_MMD_LOSS_INDEP
    else:
        op = OP_MMD_LOSS_GRAD if with_grad else OP_MMD_LOSS
    flags = (MMD_UNBIASED if unbiased else 0) | (MMD_SQRT if sqrt_loss else 0) | (MMD_INDEP if indep else 0)
    ws = _WS.get(lib.iqp_workspace_bytes(op, n, m, l, s, N, prec), G.device)
    loss = torch.empty(1, dtype=torch.float64, device=G.device)
    st = ctypes.c_void_p(_stream(G.device))
    args = (n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(X), N, X.shape[1],
            _ptr(th), prec, flags)
    if with_grad:
        grad = torch.empty(m, dtype=torch.float64, device=G.device)
        check(lib.iqp_mmd_loss_grad(*args, _ptr(loss), _ptr(grad), _ptr(ws), ws.numel(), st), "iqp_mmd_loss_grad")
        return loss[0], grad
    check(lib.iqp_mmd_loss(*args, _ptr(loss), _ptr(ws), ws.numel(), st), "iqp_mmd_loss")
    return loss[0], None


class _MmdFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, Z, X, n, precision, unbiased, sqrt_loss, indep):
        loss, grad = mmd_loss_raw(n, theta, G, A, Z, X, precision, unbiased, with_grad=theta.requires_grad,
                                  sqrt_loss=sqrt_loss, indep=indep)
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=theta.device))
        ctx.theta_dtype = theta.dtype
        return loss

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g.to(torch.float64) * grad).to(ctx.theta_dtype), None, None, None, None, None, None, None, None, None


def mmd_loss(theta, G, A, Z, X, n: int, precision="split_bf16", unbiased=True, sqrt_loss=False, indep=False):
    """MMD^2 estimate (float64 scalar tensor), differentiable in theta: the loss
    and its gradient come from one library call (its statistics pass keeps Phi
    for the gradient pass; the plain FP32 form and independent batches
    recompute it). sqrt_loss returns sqrt(max(MMD^2, 0)); indep uses one
    sample batch per observable (Z with l * s rows)."""
    return _MmdFn.apply(theta, G, A, Z, X, n, precision, unbiased, sqrt_loss, indep)


# ------------------------------------------------------ independent batches

def expval_indep_raw(n, theta, G, A, Z):
    """(expval, std_err) with one sample batch per observable: observable a
    uses rows a*s..a*s+s-1 of Z (Z has l * s rows). No autograd."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l = G.shape[0], A.shape[0]
    if Z.shape[0] % l:
        raise ValueError("Z must have l * s rows")
    s = Z.shape[0] // l
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_EXPVAL_INDEP, n, m, l, s, 0, SPARSE_FP32), G.device)
    ev = torch.empty(l, dtype=torch.float64, device=G.device)
    se = torch.empty(l, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval_indep(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1], _ptr(th),
                               _ptr(ev), _ptr(se), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(G.device))),
          "iqp_expval_indep")
    return ev, se


def expval_indep_grad(n, theta, G, A, Z, alpha, beta=None) -> torch.Tensor:
    """Gradient of the independent-batch estimator (alpha/beta as in expval_grad)."""
    for t, nm in ((G, "G"), (A, "A"), (Z, "Z")):
        _bits(t, nm)
    th = _theta32(theta)
    m, l = G.shape[0], A.shape[0]
    s = Z.shape[0] // l
    al = alpha.detach().to(device=G.device, dtype=torch.float64).contiguous()
    be = None if beta is None else beta.detach().to(device=G.device, dtype=torch.float64).contiguous()
    lib = _lib.load()
    ws = _WS.get(lib.iqp_workspace_bytes(OP_EXPVAL_INDEP_GRAD, n, m, l, s, 0, SPARSE_FP32), G.device)
    grad = torch.empty(m, dtype=torch.float64, device=G.device)
    check(lib.iqp_expval_indep_grad(n, _ptr(G), m, G.shape[1], _ptr(A), l, A.shape[1], _ptr(Z), s, Z.shape[1],
                                    _ptr(th), _ptr(al), _ptr(be), _ptr(grad), _ptr(ws), ws.numel(),
                                    ctypes.c_void_p(_stream(G.device))), "iqp_expval_indep_grad")
    return grad


class _ExpvalIndepFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, G, A, Z, n):
        ev, se = expval_indep_raw(n, theta, G, A, Z)
        ctx.save_for_backward(theta, G, A, Z)
        ctx.n = n
        ctx.mark_non_differentiable(se)
        return ev, se

    @staticmethod
    def backward(ctx, g_ev, g_se):
        theta, G, A, Z = ctx.saved_tensors
        if g_ev is None:
            return (None,) * 5
        s = Z.shape[0] // A.shape[0]
        grad = expval_indep_grad(ctx.n, theta, G, A, Z, -g_ev.to(torch.float64) / s, None)
        return grad.to(theta.dtype), None, None, None, None


def expval_indep(theta, G, A, Z, n: int):
    """indep_estimates: <Z_a> and standard errors with one sample batch per
    observable (uncorrelated estimates), differentiable in theta."""
    return _ExpvalIndepFn.apply(theta, G, A, Z, n)


# ----------------------------------------------- shared-parameter gates

def _start_dev(start, device) -> torch.Tensor:
    st = torch.as_tensor(start, dtype=torch.int64)
    return st.to(device).contiguous()


class _ExpandFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta_p, start, m):
        th = _theta32(theta_p)
        out = torch.empty(m, dtype=torch.float32, device=th.device)
        check(_lib.load().iqp_expand_params(_ptr(th), th.shape[0], _ptr(start), _ptr(out), m,
                                            ctypes.c_void_p(_stream(th.device))), "iqp_expand_params")
        ctx.save_for_backward(start)
        ctx.np, ctx.m, ctx.dtype = th.shape[0], m, theta_p.dtype
        return out

    @staticmethod
    def backward(ctx, g):
        (start,) = ctx.saved_tensors
        gg = g.detach().to(torch.float64).contiguous()
        out = torch.empty(ctx.np, dtype=torch.float64, device=gg.device)
        check(_lib.load().iqp_reduce_params(_ptr(gg), ctx.m, _ptr(start), ctx.np, _ptr(out),
                                            ctypes.c_void_p(_stream(gg.device))), "iqp_reduce_params")
        return out.to(ctx.dtype), None, None


def expand_params(theta_p, start, m: int):
    """Shared-parameter gates (Sec. 3.1.1): per-generator parameters from one
    parameter per gate; gate p owns generator rows start[p]..start[p+1]-1.
    Differentiable: the gradient of a gate is the sum over its generators."""
    return _ExpandFn.apply(theta_p, _start_dev(start, theta_p.device), m)


# ---------------------------------------------------------- wires, RNG

def embed_bits(src: torch.Tensor, nw: int, wires, n: int) -> torch.Tensor:
    """Rows on nw wire qubits -> rows on n qubits (bit k -> qubit wires[k])."""
    _bits(src, "src")
    w = torch.as_tensor(wires, dtype=torch.int32).to(src.device).contiguous()
    ld = words_per_row(n)
    out = torch.empty(src.shape[0], ld, dtype=torch.int64, device=src.device)
    check(_lib.load().iqp_embed_bits(_ptr(src), src.shape[0], src.shape[1], _ptr(w), nw, _ptr(out), ld, n,
                                     ctypes.c_void_p(_stream(src.device))), "iqp_embed_bits")
    return out


def words_per_row(n: int) -> int:
    w = max(1, (n + 63) // 64)
    return w + (w & 1)


def _bits_out(out, rows, ld, device):
    if out is None:
        return torch.empty(rows, ld, dtype=torch.int64, device=device)
    if not (out.is_cuda and out.dtype == torch.int64 and out.shape == (rows, ld) and out.is_contiguous()):
        raise ValueError(f"out must be a contiguous ({rows}, {ld}) int64 CUDA tensor")
    return out


def uniform_bits(seed: int, stream: int, rows: int, n: int, device="cuda", out=None) -> torch.Tensor:
    """Uniform bitstrings drawn on the device (same bits as
    inputs.uniform_bits(Rng(seed), rows, n, stream)), into `out` if given."""
    ld = words_per_row(n)
    out = _bits_out(out, rows, ld, device)
    check(_lib.load().iqp_uniform_bits(seed & (2 ** 64 - 1), stream & (2 ** 64 - 1), rows, n, _ptr(out), ld,
                                       ctypes.c_void_p(_stream(device))), "iqp_uniform_bits")
    return out


def bernoulli_bits(seed: int, stream: int, rows: int, n: int, p: float, device="cuda", out=None) -> torch.Tensor:
    """Bernoulli(p) bits drawn on the device (same bits as
    inputs.bernoulli_bits(Rng(seed), rows, n, p, stream)), into `out` if given."""
    ld = words_per_row(n)
    out = _bits_out(out, rows, ld, device)
    check(_lib.load().iqp_bernoulli_bits(seed & (2 ** 64 - 1), stream & (2 ** 64 - 1), rows, n, float(p),
                                         _ptr(out), ld, ctypes.c_void_p(_stream(device))), "iqp_bernoulli_bits")
    return out


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
    device = _resolve("cuda" if device is None else device)
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
