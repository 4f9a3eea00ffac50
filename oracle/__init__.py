"""FP64 CPU oracle for the IQP Monte-Carlo estimator (ctypes wrapper).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm may import this package. The CUDA path neither
imports nor links it, and it imports nothing from the CUDA path.

The arithmetic lives in iqp_oracle.c (plain C, double precision). This file
builds it with gcc and marshals numpy arrays; it computes nothing itself.
Each function documents which equation of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iqp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile iqp_oracle.c -> liboracle.so (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        mat = [p, i64, i64]
        sig = {
            "oracle_parity": [i64] + mat + mat + [p],
            "oracle_expval": [i64] + mat * 3 + [p, p, p, p, p],
            "oracle_expval_grad": [i64] + mat * 3 + [p, p, p, p],
            "oracle_data_parity_sum": [i64] + mat + mat + [p],
            "oracle_mmd_loss": [i64] + mat * 4 + [p, ctypes.c_int, p, p, p],
            "oracle_exact_expval": [i64] + mat * 2 + [p, p],
            "oracle_statevector_probs": [i64] + mat + [p, p],
            "oracle_statevector_expval": [i64] + mat * 2 + [p, p],
            "oracle_subset_expansion": [i64] + mat * 2 + [p, p],
            "oracle_bitflip_expval": [i64] + mat * 2 + [p, p],
            "oracle_bitflip_grad": [i64] + mat * 2 + [p, p, p],
            "oracle_mmd_loss_sqrt": [i64] + mat * 4 + [p, ctypes.c_int, p, p],
            "oracle_mmd_loss_ex": [i64] + mat * 4 + [p, ctypes.c_int, p, p, p],
            "oracle_expand_params": [p, p, i64, p],
            "oracle_reduce_params": [p, p, i64, p],
            "oracle_embed_bits": [p, i64, i64, p, i64, p, i64],
            "oracle_expval_indep": [i64] + mat * 3 + [p, p, p, p, p],
            "oracle_expval_indep_grad": [i64] + mat * 3 + [p, p, p, p],
            "oracle_set_threads": [ctypes.c_int],
            "oracle_max_threads": [],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int if name == "oracle_max_threads" else None
        _lib = lib
    return _lib


def _w(a):
    """Packed bit matrix -> (contiguous uint64 array, pointer, rows, ld)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.ndim == 1:
        a = a.reshape(1, -1)
    return a, a.ctypes.data, a.shape[0], a.shape[1]


def _d(x, n=None):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return x


def set_threads(t: int):
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return _load().oracle_max_threads()


def parity(n, R, G):
    """P[r, j] = (R_r . g_j) mod 2 as uint8 (A.G^T or Z.G^T mod 2, Sec. 2.2)."""
    lib = _load()
    R, pr, rows, ldr = _w(R)
    G, pg, m, ldg = _w(G)
    P = np.empty((rows, m), dtype=np.uint8)
    lib.oracle_parity(n, pr, rows, ldr, pg, m, ldg, P.ctypes.data)
    return P


def expval(n, G, A, Z, theta):
    """Estimator of eq. expvalsample on the given samples: returns
    (expval, std_err, S1, S2), each float64[l]; theta is cast to float64."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, s, ldz = _w(Z)
    th = _d(theta)
    assert th.shape[0] == m
    ev, se, s1, s2 = (np.empty(l) for _ in range(4))
    lib.oracle_expval(n, pg, m, ldg, pa, l, lda, pz, s, ldz, th.ctypes.data,
                      ev.ctypes.data, se.ctypes.data, s1.ctypes.data, s2.ctypes.data)
    return ev, se, s1, s2


def expval_grad(n, G, A, Z, theta, alpha, beta=None):
    """grad_j = sum_a sum_i sin(Phi)(alpha_a + beta_a cos Phi) 2 P_A[a,j] S_Z[i,j]."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, s, ldz = _w(Z)
    th = _d(theta)
    al = _d(alpha)
    be = _d(beta) if beta is not None else None
    g = np.empty(m)
    lib.oracle_expval_grad(n, pg, m, ldg, pa, l, lda, pz, s, ldz, th.ctypes.data, al.ctypes.data,
                           be.ctypes.data if be is not None else None, g.ctypes.data)
    return g


def data_parity_sum(n, A, X):
    """T_a = sum_x (-1)^{a.x} (int64[l])."""
    lib = _load()
    A, pa, l, lda = _w(A)
    X, px, N, ldx = _w(X)
    T = np.empty(l, dtype=np.int64)
    lib.oracle_data_parity_sum(n, pa, l, lda, px, N, ldx, T.ctypes.data)
    return T


def mmd_loss(n, G, A, Z, X, theta, unbiased=True, grad=False):
    """MMD^2 estimate of eq. mmd_estimate: returns (loss, terms[l], grad[m] or None)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, s, ldz = _w(Z)
    X, px, N, ldx = _w(X)
    th = _d(theta)
    loss = ctypes.c_double(0.0)
    terms = np.empty(l)
    g = np.empty(m) if grad else None
    lib.oracle_mmd_loss(n, pg, m, ldg, pa, l, lda, pz, s, ldz, px, N, ldx, th.ctypes.data,
                        1 if unbiased else 0, ctypes.addressof(loss), terms.ctypes.data,
                        g.ctypes.data if g is not None else None)
    return loss.value, terms, g


def exact_expval(n, G, A, theta):
    """<Z_a> by enumerating all 2^n samples (eq. op_expval), n <= 24."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    out = np.empty(l)
    lib.oracle_exact_expval(n, pg, m, ldg, pa, l, lda, _d(theta).ctypes.data, out.ctypes.data)
    return out


def statevector_probs(n, G, theta):
    """|<x|U(theta)|0>|^2 for all x (index bit q = qubit q)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    pr = np.empty(1 << n)
    lib.oracle_statevector_probs(n, pg, m, ldg, _d(theta).ctypes.data, pr.ctypes.data)
    return pr


def statevector_expval(n, G, A, theta):
    """<Z_a> from the statevector (eq. expvals)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    out = np.empty(l)
    lib.oracle_statevector_expval(n, pg, m, ldg, pa, l, lda, _d(theta).ctypes.data, out.ctypes.data)
    return out


def subset_expansion(n, G, A, theta):
    """<Z_a> by the subset expansion of eq. expval_intefere (brute force)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    out = np.empty(l)
    lib.oracle_subset_expansion(n, pg, m, ldg, pa, l, lda, _d(theta).ctypes.data, out.ctypes.data)
    return out


def bitflip_expval(n, G, A, theta):
    """Stochastic bitflip circuit <Z_a> = prod_{j in J_a} cos(2 theta_j)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    out = np.empty(l)
    lib.oracle_bitflip_expval(n, pg, m, ldg, pa, l, lda, _d(theta).ctypes.data, out.ctypes.data)
    return out


def bitflip_grad(n, G, A, theta, w):
    """d/dtheta of sum_a w_a prod_{j in J_a} cos(2 theta_j) (product rule)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    g = np.empty(m)
    lib.oracle_bitflip_grad(n, pg, m, ldg, pa, l, lda, _d(theta).ctypes.data, _d(w).ctypes.data, g.ctypes.data)
    return g


def mmd_loss_sqrt(n, G, A, Z, X, theta, unbiased=True, grad=False):
    """sqrt_loss form of the MMD loss: (sqrt(MMD^2 estimate), grad or None)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, s, ldz = _w(Z)
    X, px, N, ldx = _w(X)
    loss = ctypes.c_double(0.0)
    g = np.empty(m) if grad else None
    lib.oracle_mmd_loss_sqrt(n, pg, m, ldg, pa, l, lda, pz, s, ldz, px, N, ldx, _d(theta).ctypes.data,
                             1 if unbiased else 0, ctypes.addressof(loss), g.ctypes.data if g is not None else None)
    return loss.value, g


def mmd_loss_ex(n, G, A, Z, X, theta, unbiased=True, sqrt_loss=False, indep=False, grad=False):
    """MMD loss with the API options: sqrt_loss, indep (Z has l * s rows, one
    batch per observable). Returns (loss, terms[l], grad[m] or None)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, zr, ldz = _w(Z)
    X, px, N, ldx = _w(X)
    s = zr // l if indep else zr
    flags = (1 if unbiased else 0) | (2 if sqrt_loss else 0) | (4 if indep else 0)
    loss = ctypes.c_double(0.0)
    terms = np.empty(l)
    g = np.empty(m) if grad else None
    lib.oracle_mmd_loss_ex(n, pg, m, ldg, pa, l, lda, pz, s, ldz, px, N, ldx, _d(theta).ctypes.data, flags,
                           ctypes.addressof(loss), terms.ctypes.data, g.ctypes.data if g is not None else None)
    return loss.value, terms, g


def expand_params(theta_p, start):
    """Per-generator parameters of shared-parameter gates (gate p owns
    generators start[p]..start[p+1]-1)."""
    lib = _load()
    th = _d(theta_p)
    st = np.ascontiguousarray(start, dtype=np.int64)
    out = np.empty(int(st[-1]))
    lib.oracle_expand_params(th.ctypes.data, st.ctypes.data, th.shape[0], out.ctypes.data)
    return out


def reduce_params(grad_gen, start):
    """Gradient per shared parameter: sum over the gate's generators."""
    lib = _load()
    g = _d(grad_gen)
    st = np.ascontiguousarray(start, dtype=np.int64)
    out = np.empty(st.shape[0] - 1)
    lib.oracle_reduce_params(g.ctypes.data, st.ctypes.data, out.shape[0], out.ctypes.data)
    return out


def embed_bits(src, nw, wires, n):
    """Rows on `nw` wire qubits -> rows on n qubits (bit k -> qubit wires[k])."""
    lib = _load()
    S, ps, rows, lds = _w(src)
    wi = np.ascontiguousarray(wires, dtype=np.int64)
    assert wi.shape[0] == nw
    ld = max(1, (n + 63) // 64)
    ld += ld & 1
    out = np.empty((rows, ld), dtype=np.uint64)
    lib.oracle_embed_bits(ps, rows, lds, wi.ctypes.data, nw, out.ctypes.data, ld)
    return out


def expval_indep(n, G, A, Z, theta):
    """Independent-batch estimator: observable a uses Z rows a*s..a*s+s-1.
    Returns (expval, std_err, S1, S2)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, ls, ldz = _w(Z)
    assert ls % l == 0
    s = ls // l
    ev, se, s1, s2 = (np.empty(l) for _ in range(4))
    lib.oracle_expval_indep(n, pg, m, ldg, pa, l, lda, pz, s, ldz, _d(theta).ctypes.data,
                            ev.ctypes.data, se.ctypes.data, s1.ctypes.data, s2.ctypes.data)
    return ev, se, s1, s2


def expval_indep_grad(n, G, A, Z, theta, alpha, beta=None):
    """Gradient of the independent-batch estimator (alpha/beta as in expval_grad)."""
    lib = _load()
    G, pg, m, ldg = _w(G)
    A, pa, l, lda = _w(A)
    Z, pz, ls, ldz = _w(Z)
    s = ls // l
    al = _d(alpha)
    be = _d(beta) if beta is not None else None
    g = np.empty(m)
    lib.oracle_expval_indep_grad(n, pg, m, ldg, pa, l, lda, pz, s, ldz, _d(theta).ctypes.data, al.ctypes.data,
                                 be.ctypes.data if be is not None else None, g.ctypes.data)
    return g


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
