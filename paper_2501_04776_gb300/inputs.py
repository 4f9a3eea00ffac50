"""Seeded synthetic inputs for the IQP estimator: generators G, observables A,
samples Z, data X and parameters theta.

This module holds the random-number generator, the bit-packing format of the
C ABI and the workload recipes. It holds none of the estimator's arithmetic:
no parities, phases, cosines or losses. Both the CUDA path and the CPU oracle
consume what it produces, so they always see identical bits and parameters.

Bit format (the C ABI's): a binary matrix with `rows` rows and `n` columns is
stored as uint64 words, row-major, `ld` words per row with `ld` even (16-byte
rows), LSB-first: bit b of word w is column 64*w + b. Padding bits are zero.

Random numbers come from a counter-based splitmix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value k of
stream t under seed S is mix(S*PHI + t*PSI + (k+1)*GAMMA). Uniform doubles take
the top 53 bits; normals use Box-Muller. The paper draws with JAX keys, which
cannot be reproduced here; any uniform source serves the estimator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_PHI = np.uint64(0xD1B54A32D192ED03)
_PSI = np.uint64(0xAEF17502108EF2D9)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Stafford variant 13), vectorised, wrapping uint64."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


class Rng:
    """Counter-based splitmix64 streams. Every call names its stream, so draws
    do not depend on call order."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def u64(self, count: int, stream: int, offset: int = 0) -> np.ndarray:
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            base = self.seed * _PHI + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _PSI
            return _mix(base + k * _GAMMA)

    def uniform(self, count: int, stream: int, offset: int = 0) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(count, stream, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, count: int, stream: int) -> np.ndarray:
        """Standard normals by Box-Muller on pairs of uniforms."""
        half = (count + 1) // 2
        u = self.uniform(2 * half, stream)
        u1 = 1.0 - u[0::2]  # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * half)
        out[0::2] = r * np.cos(2.0 * math.pi * u2)
        out[1::2] = r * np.sin(2.0 * math.pi * u2)
        return out[:count]

    def integers(self, count: int, high, stream: int) -> np.ndarray:
        """Integers in [0, high) (high may be an array), by 128-bit-free
        multiply-shift on 32-bit halves; bias below 2^-32 for high < 2^32."""
        u = (self.u64(count, stream) >> np.uint64(32)).astype(np.uint64)
        high = np.asarray(high, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return ((u * high) >> np.uint64(32)).astype(np.int64)


# ---------------------------------------------------------------- bit format

def words_per_row(n: int) -> int:
    """ld of the C ABI: ceil(n/64) rounded up to even (16-byte rows)."""
    w = max(1, (n + 63) // 64)
    return w + (w & 1)


def pack_bits(bits: np.ndarray, ld: int | None = None) -> np.ndarray:
    """(rows, n) array of 0/1 -> (rows, ld) uint64, LSB-first, zero padding."""
    bits = np.asarray(bits, dtype=np.uint8)
    rows, n = bits.shape
    ld = words_per_row(n) if ld is None else ld
    padded = np.zeros((rows, ld * 64), dtype=np.uint8)
    padded[:, :n] = bits & 1
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u8").reshape(rows, ld).astype(np.uint64)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_bits: (rows, ld) uint64 -> (rows, n) uint8."""
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    rows = words.shape[0]
    by = words.astype("<u8").view(np.uint8).reshape(rows, -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n]


def pack_index_lists(gates, n: int) -> np.ndarray:
    """Generators given as lists of qubit indices (the paper's gate format)
    -> packed rows."""
    ld = words_per_row(n)
    out = np.zeros((len(gates), ld), dtype=np.uint64)
    for r, g in enumerate(gates):
        for q in g:
            out[r, q >> 6] ^= np.uint64(1) << np.uint64(q & 63)
    return out


def local_gates(n: int) -> list[list[int]]:
    """All one- and two-body generators in the paper's order: [0], [1], ...,
    [n-1], then pairs (q1 < q2) in lexicographic order (Sec. 3.1.1)."""
    return [[q] for q in range(n)] + [[a, b] for a in range(n) for b in range(a + 1, n)]


def local_gates_packed(n: int) -> np.ndarray:
    """local_gates(n) packed, built without Python loops over pairs."""
    ld = words_per_row(n)
    m = n + n * (n - 1) // 2
    out = np.zeros((m, ld), dtype=np.uint64)
    q = np.arange(n)
    out[q, q >> 6] = np.uint64(1) << (q & 63).astype(np.uint64)
    a, b = np.triu_indices(n, k=1)  # row-major: lexicographic pairs
    rows = n + np.arange(a.size)
    out[rows, a >> 6] |= np.uint64(1) << (a & 63).astype(np.uint64)
    out[rows, b >> 6] |= np.uint64(1) << (b & 63).astype(np.uint64)
    return out


# ------------------------------------------------------------ random objects

def uniform_bits(rng: Rng, rows: int, n: int, stream: int) -> np.ndarray:
    """Uniform bitstrings (samples z ~ U{0,1}^n), packed."""
    ld = words_per_row(n)
    w = rng.u64(rows * ld, stream).reshape(rows, ld)
    full, rem = divmod(n, 64)
    if full < ld:
        w[:, full + (1 if rem else 0):] = 0
        if rem:
            w[:, full] &= np.uint64((1 << rem) - 1)
    return w


def bernoulli_bits(rng: Rng, rows: int, n: int, p: float, stream: int,
                   nonzero: bool = False, chunk_rows: int = 2048) -> np.ndarray:
    """Rows of i.i.d. Bernoulli(p) bits, packed. With nonzero=True an all-zero
    row is redrawn (from further counters of the same stream)."""
    ld = words_per_row(n)
    out = np.zeros((rows, ld), dtype=np.uint64)
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        u = rng.uniform((r1 - r0) * n, stream, offset=r0 * n).reshape(r1 - r0, n)
        out[r0:r1] = pack_bits(u < p, ld)
    if nonzero:
        redraw = 0
        for r in range(rows):
            while not out[r].any():
                redraw += 1
                u = rng.uniform(n, stream, offset=rows * n + redraw * n)
                out[r] = pack_bits((u < p)[None, :], ld)[0]
    return out


def random_k_body(rng: Rng, m: int, n: int, ks, stream: int) -> np.ndarray:
    """m generators; each picks k uniformly from `ks`, then k distinct qubits
    uniformly (skip-over sampling, k <= 3)."""
    ks = np.asarray(ks)
    assert ks.max() <= 3 and n >= ks.max()
    k = ks[rng.integers(m, ks.size, stream)]
    r0 = rng.integers(m, n, stream + 1)
    r1 = rng.integers(m, max(n - 1, 1), stream + 2)
    r2 = rng.integers(m, max(n - 2, 1), stream + 3)
    q0 = r0
    q1 = r1 + (r1 >= q0)
    lo, hi = np.minimum(q0, q1), np.maximum(q0, q1)
    q2 = r2 + (r2 >= lo)
    q2 = q2 + (q2 >= hi)
    ld = words_per_row(n)
    out = np.zeros((m, ld), dtype=np.uint64)
    rows = np.arange(m)
    for q, use in ((q0, k >= 1), (q1, k >= 2), (q2, k >= 3)):
        rr, qq = rows[use], q[use]
        np.bitwise_or.at(out, (rr, qq >> 6), np.uint64(1) << (qq & 63).astype(np.uint64))
    return out


def prototype_data(rng: Rng, N: int, n: int, n_proto: int, flip: float, stream: int) -> np.ndarray:
    """N data rows: each copies one of n_proto uniform prototype bitstrings
    (chosen uniformly) and flips each bit independently with probability flip."""
    ld = words_per_row(n)
    protos = uniform_bits(rng, n_proto, n, stream)
    pick = rng.integers(N, n_proto, stream + 1)
    flips = bernoulli_bits(rng, N, n, flip, stream + 2)
    return protos[pick] ^ flips


def p_sigma(sigma2: float) -> float:
    """Bit probability of the observable distribution for a Gaussian kernel of
    bandwidth sigma on Hamming distance (bits i.i.d. Bernoulli(p_sigma))."""
    return 0.5 * (1.0 - math.exp(-1.0 / (2.0 * sigma2)))


# ----------------------------------------------------------------- workloads

@dataclass
class Problem:
    """One seeded instance: packed G (m x ldn), A (l x ldn), Z (s x ldn),
    optional X (N x ldn), theta (fp32[m]) and optional loss weights w."""
    name: str
    n: int
    G: np.ndarray
    A: np.ndarray
    Z: np.ndarray
    theta: np.ndarray
    X: np.ndarray | None = None
    w: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def m(self): return self.G.shape[0]
    @property
    def l(self): return self.A.shape[0]
    @property
    def s(self): return self.Z.shape[0]


def tiny_local(seed: int = 1, n: int = 8, l: int = 64, s: int = 1024) -> Problem:
    """n=8, all one- and two-body generators (m=36), theta ~ N(0, 0.3^2) fp32,
    64 nonzero observables with Bernoulli(0.5) bits, 1024 uniform samples."""
    rng = Rng(seed)
    G = local_gates_packed(n)
    theta = (0.3 * rng.normal(G.shape[0], 10)).astype(np.float32)
    A = bernoulli_bits(rng, l, n, 0.5, 20, nonzero=True)
    Z = uniform_bits(rng, s, n, 30)
    return Problem("local-n8-m36-l64-s1024", n, G, A, Z, theta)


def local300(seed: int = 2, n: int = 300, l: int = 1000, s: int = 10000) -> Problem:
    """n=300, all one- and two-body generators (m=45150), theta ~ N(0, 0.01^2),
    1000 observables with Bernoulli(0.1) bits, 10000 samples, loss weights
    w ~ N(0, 1)."""
    rng = Rng(seed)
    G = local_gates_packed(n)
    theta = (0.01 * rng.normal(G.shape[0], 10)).astype(np.float32)
    A = bernoulli_bits(rng, l, n, 0.1, 20)
    Z = uniform_bits(rng, s, n, 30)
    w = rng.normal(l, 40)
    return Problem(f"local-n{n}-m{G.shape[0]}-l{l}-s{s}", n, G, A, Z, theta, w=w)


def random_gates(seed: int = 3, n: int = 1000, m: int = 100_000, l: int = 10_000,
                 s: int = 10_000) -> Problem:
    """m random generators on k in {1,2,3} distinct qubits, theta ~ U(-0.05,
    0.05), observables with Bernoulli(0.05) bits, uniform samples."""
    rng = Rng(seed)
    G = random_k_body(rng, m, n, [1, 2, 3], 10)
    theta = (0.1 * rng.uniform(m, 20) - 0.05).astype(np.float32)
    A = bernoulli_bits(rng, l, n, 0.05, 30)
    Z = uniform_bits(rng, s, n, 40)
    w = rng.normal(l, 50)
    return Problem(f"random-n{n}-m{m}-l{l}-s{s}", n, G, A, Z, theta, w=w)


def mmd_training(seed: int = 4, n: int = 1000, l: int = 2000, s: int = 5000,
                 N: int = 10_000, m: int | None = None) -> Problem:
    """MMD training workload: all one- and two-body generators on n qubits
    (m = n(n+1)/2), data = N rows from 8 uniform prototypes with 5% bit flips,
    observables with Bernoulli(p_sigma) bits for sigma = sqrt(n)/4, initial
    theta ~ N(0, 0.01^2). `m` truncates the generator list (small tests)."""
    rng = Rng(seed)
    G = local_gates_packed(n)
    if m is not None:
        G = G[:m]
    theta = (0.01 * rng.normal(G.shape[0], 10)).astype(np.float32)
    sigma2 = n / 16.0
    ps = p_sigma(sigma2)
    A = bernoulli_bits(rng, l, n, ps, 20)
    Z = uniform_bits(rng, s, n, 30)
    X = prototype_data(rng, N, n, 8, 0.05, 40)
    return Problem(f"mmd-n{n}-m{G.shape[0]}-l{l}-s{s}-N{N}", n, G, A, Z, theta, X=X,
                   extra={"sigma2": sigma2, "p_sigma": ps})


def million_gates(seed: int = 5, n: int = 5000, m: int = 1_000_000, l: int = 4096,
                  s: int = 16384) -> Problem:
    """n=5000, one million random one- and two-body generators, theta ~
    N(0, 0.005^2), observables with Bernoulli(0.01) bits, 16384 samples."""
    rng = Rng(seed)
    G = random_k_body(rng, m, n, [1, 2], 10)
    theta = (0.005 * rng.normal(m, 20)).astype(np.float32)
    A = bernoulli_bits(rng, l, n, 0.01, 30)
    Z = uniform_bits(rng, s, n, 40)
    w = rng.normal(l, 50)
    return Problem(f"random-n{n}-m{m}-l{l}-s{s}", n, G, A, Z, theta, w=w)


def fresh_samples(seed: int, step: int, s: int, n: int) -> np.ndarray:
    """A new sample batch per optimisation step (new Z every step, Sec. 2.4)."""
    return uniform_bits(Rng(seed), s, n, 1000 + 2 * step)


def fresh_observables(seed: int, step: int, l: int, n: int, p: float) -> np.ndarray:
    """A new observable batch per step (ops drawn inside the MMD loss)."""
    return bernoulli_bits(Rng(seed), l, n, p, 1001 + 2 * step)
