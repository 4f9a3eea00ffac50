"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself: the one-gate closed form, product forms (eq.
expval_bitflip when no subset of J_a XORs to zero), three independent exact
evaluations (enumeration of eq. op_expval, a statevector built from the gate
action of Sec. 2.5, the subset expansion of eq. expval_intefere), the MC error
bound, a hand-derived standard error, central finite differences, numpy
brute force for GF(2) products, pair-mean U-statistics, the kernel form of
MMD^2 (eq. mmd_loss) against its observable form (eq. mmd_estimate), and the
per-qubit/per-pair regrouping of the phase and its gradient for generators of
weight <= 2.

All CPU; no GPU, no CUDA extension.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_04776_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def bits_of(words, n):
    return I.unpack_bits(words, n).astype(np.int64)


def all_strings(n):
    return I.pack_bits(np.array(list(itertools.product([0, 1], repeat=n)))[:, ::-1])


# ------------------------------------------------------------------ parities

def test_parity_matches_numpy_gf2_product():
    rng = I.Rng(11)
    n = 203  # four words, ragged
    R = I.bernoulli_bits(rng, 37, n, 0.5, 1)
    G = I.bernoulli_bits(rng, 53, n, 0.3, 2)
    want = (bits_of(R, n) @ bits_of(G, n).T) % 2
    got = oracle.parity(n, R, G)
    assert np.array_equal(got, want.astype(np.uint8))


def test_data_parity_sum_matches_numpy():
    rng = I.Rng(12)
    n = 70
    A = I.bernoulli_bits(rng, 9, n, 0.2, 1)
    X = I.uniform_bits(rng, 41, n, 2)
    par = (bits_of(A, n) @ bits_of(X, n).T) % 2
    want = (1 - 2 * par).sum(axis=1)
    assert np.array_equal(oracle.data_parity_sum(n, A, X), want)


# ------------------------------------------------------------ exact forms

@pytest.mark.parametrize("theta", [0.0, 0.1, -0.37, 0.785, 1.3, 2.9])
def test_single_gate_is_cos_2theta(theta):
    """One gate exp(i theta X) on one qubit: <Z> = cos(2 theta)."""
    G = I.pack_index_lists([[0]], 1)
    A = I.pack_index_lists([[0]], 1)
    th = np.array([theta])
    want = math.cos(2 * theta)
    for got in (oracle.exact_expval(1, G, A, th), oracle.statevector_expval(1, G, A, th),
                oracle.subset_expansion(1, G, A, th)):
        assert abs(got[0] - want) < 1e-14
    # Every sample of the estimator gives cos(+-2 theta) = cos(2 theta): SE = 0.
    ev, se, _, _ = oracle.expval(1, G, A, all_strings(1), th)
    assert abs(ev[0] - want) < 1e-15 and se[0] < 1e-15


def test_theta_zero_and_trivial_observables_give_one():
    p = I.tiny_local(seed=3)
    th0 = np.zeros(p.m)
    ev, se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, th0)
    assert np.all(ev == 1.0) and np.all(se == 0.0)
    # a = 0, and an observable commuting with every generator (even overlap
    # with each one-body and two-body gate is impossible unless a = 0, so use
    # generators restricted to qubits outside a's support).
    G = I.pack_index_lists([[0, 1], [2], [1, 2], [2, 3]], 6)
    A = I.pack_index_lists([[], [4, 5]], 6)
    th = np.array([0.3, -0.8, 1.1, 0.4])
    ev, se, _, _ = oracle.expval(6, G, A, all_strings(6), th)
    assert np.all(ev == 1.0) and np.all(se == 0.0)


def test_one_body_generators_product_form():
    """One-body generators: gates on the same qubit add their angles, so
    <Z_a> = prod_{q in a} cos(2 Theta_q), Theta_q = sum of theta on qubit q."""
    rng = I.Rng(21)
    n = 6
    qubits = rng.integers(14, n, 1)
    G = I.pack_index_lists([[int(q)] for q in qubits], n)
    th = rng.normal(14, 2) * 0.7
    A = I.bernoulli_bits(rng, 20, n, 0.5, 3)
    Theta = np.zeros(n)
    np.add.at(Theta, qubits, th)
    want = np.array([np.prod(np.cos(2 * Theta[row.astype(bool)])) for row in bits_of(A, n)])
    for got in (oracle.exact_expval(n, G, A, th), oracle.statevector_expval(n, G, A, th),
                oracle.subset_expansion(n, G, A, th)):
        assert np.max(np.abs(got - want)) < 1e-12


def chain_gates(n):
    """Generators X_q X_{q+1}: linearly independent over GF(2), so no subset of
    any J_a XORs to zero and eq. expval_intefere reduces to its product term."""
    return I.pack_index_lists([[q, q + 1] for q in range(n - 1)], n)


def test_independent_generators_product_form_exact():
    rng = I.Rng(22)
    n = 10
    G = chain_gates(n)
    th = rng.normal(n - 1, 1) * 0.5
    A = I.bernoulli_bits(rng, 30, n, 0.5, 2)
    Gb = bits_of(G, n)
    want = np.array([np.prod(np.cos(2 * th[(Gb @ a) % 2 == 1])) for a in bits_of(A, n)])
    assert np.max(np.abs(oracle.exact_expval(n, G, A, th) - want)) < 1e-12
    assert np.max(np.abs(oracle.statevector_expval(n, G, A, th) - want)) < 1e-12
    assert np.max(np.abs(oracle.bitflip_expval(n, G, A, th) - want)) < 1e-12


def test_independent_generators_mc_at_300_qubits():
    """Closed form at n=300: the MC estimate lies within 4 standard errors."""
    rng = I.Rng(23)
    n = 300
    G = chain_gates(n)
    th = (rng.normal(n - 1, 1) * 0.05)
    A = I.bernoulli_bits(rng, 24, n, 0.05, 2, nonzero=True)
    Z = I.uniform_bits(rng, 20000, n, 3)
    exact = oracle.bitflip_expval(n, G, A, th)
    ev, se, _, _ = oracle.expval(n, G, A, Z, th)
    z = np.abs(ev - exact) / np.maximum(se, 1e-300)
    assert np.all(z < 4.5), z
    assert np.mean(z) < 1.5


def test_enumeration_equals_statevector_n8_local():
    p = I.tiny_local(seed=4)
    th = p.theta.astype(np.float64)
    e = oracle.exact_expval(p.n, p.G, p.A, th)
    v = oracle.statevector_expval(p.n, p.G, p.A, th)
    assert np.max(np.abs(e - v)) < 1e-12
    # Non-trivial interference: the product (bitflip) form differs.
    b = oracle.bitflip_expval(p.n, p.G, p.A, th)
    assert np.max(np.abs(e - b)) > 1e-3


def test_subset_expansion_equals_statevector():
    rng = I.Rng(5)
    n = 5
    G = I.local_gates_packed(n)  # m = 15
    th = rng.normal(G.shape[0], 1) * 0.6
    A = I.bernoulli_bits(rng, 31, n, 0.5, 2)
    v = oracle.statevector_expval(n, G, A, th)
    s = oracle.subset_expansion(n, G, A, th)
    assert np.max(np.abs(v - s)) < 1e-12


def test_statevector_norm_and_probs():
    p = I.tiny_local(seed=6)
    pr = oracle.statevector_probs(p.n, p.G, p.theta.astype(np.float64))
    assert abs(pr.sum() - 1.0) < 1e-12 and np.all(pr >= 0)


# --------------------------------------------------------------- estimator

def test_standard_error_closed_form():
    """Two one-body gates on qubits 0 and 1, a = 11, Z = all four strings:
    cos Phi takes cos(x+y) twice and cos(x-y) twice (x=2t1, y=2t2), so the
    mean is cos x cos y and the population SD is |sin x sin y|; SE = SD/2."""
    G = I.pack_index_lists([[0], [1]], 2)
    A = I.pack_index_lists([[0, 1]], 2)
    for t1, t2 in [(0.3, -0.7), (1.2, 0.25), (-2.0, 0.9)]:
        ev, se, s1, s2 = oracle.expval(2, G, A, all_strings(2), np.array([t1, t2]))
        x, y = 2 * t1, 2 * t2
        assert abs(ev[0] - math.cos(x) * math.cos(y)) < 1e-15
        assert abs(se[0] - abs(math.sin(x) * math.sin(y)) / 2) < 1e-15
        assert abs(s1[0] - 4 * ev[0]) < 1e-14
        assert abs(s2[0] - 2 * (math.cos(x + y) ** 2 + math.cos(x - y) ** 2)) < 1e-14


def test_theta_sign_symmetry_on_fixed_samples():
    p = I.tiny_local(seed=7, s=256)
    th = p.theta.astype(np.float64)
    a = oracle.expval(p.n, p.G, p.A, p.Z, th)[0]
    b = oracle.expval(p.n, p.G, p.A, p.Z, -th)[0]
    assert np.array_equal(a, b)


def test_mc_within_three_standard_errors():
    """Unbiased MC estimate (Prop. 1): within 3 SE of the exact value for all
    but a few of 64 observables. The observables share one sample batch, so
    their errors are correlated (Sec. 2.2) and misses come in groups; the RMS
    of the standardised errors must still be near 1."""
    p = I.tiny_local(seed=1)
    th = p.theta.astype(np.float64)
    exact = oracle.exact_expval(p.n, p.G, p.A, th)
    ev, se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, th)
    z = np.abs(ev - exact) / se
    assert np.sum(z > 3) <= 3, z
    assert 0.6 < math.sqrt(np.mean(z ** 2)) < 1.4
    # Averaging over every sample string gives the exact value.
    ev_all, _, _, _ = oracle.expval(p.n, p.G, p.A, all_strings(p.n), th)
    assert np.max(np.abs(ev_all - exact)) < 1e-12


def test_standard_error_scaling_and_paper_precision():
    """SE ~ 1/sqrt(s); with phases spread over many periods Var(cos) -> 1/2, and
    the paper's precision of about 0.007 at 10000 samples appears."""
    gold = json.load(open(GOLDEN))["precision_at_10000_samples"]["value"]
    rng = I.Rng(31)
    n, m = 100, 2000
    G = I.random_k_body(rng, m, n, [1, 2, 3], 1)
    th = rng.uniform(m, 5) * 2 * math.pi
    A = I.bernoulli_bits(rng, 12, n, 0.05, 6, nonzero=True)
    Z = I.uniform_bits(rng, 10000, n, 7)
    _, se_big, _, _ = oracle.expval(n, G, A, Z, th)
    _, se_small, _, _ = oracle.expval(n, G, A, Z[:1000], th)
    ratio = se_small / se_big
    assert np.all(np.abs(ratio - math.sqrt(10)) < 0.35 * math.sqrt(10))
    assert abs(np.median(se_big) - gold) < 0.001
    assert abs(np.median(se_big) - math.sqrt(0.5 / 10000)) < 0.0006


# ----------------------------------------------------------------- gradient

def _fd(f, th, h=1e-5):
    g = np.empty_like(th)
    for j in range(th.size):
        e = np.zeros_like(th)
        e[j] = h
        g[j] = (f(th + e) - f(th - e)) / (2 * h)
    return g


def test_grad_matches_central_differences():
    """For F(theta) = -sum_a (alpha_a S1_a + beta_a S2_a / 2) the oracle's
    gradient formula must equal dF/dtheta (Sec. 2.4: deterministic in theta
    for fixed samples)."""
    rng = I.Rng(41)
    n = 6
    G = I.local_gates_packed(n)
    m = G.shape[0]
    th = rng.normal(m, 1) * 0.4
    A = I.bernoulli_bits(rng, 5, n, 0.5, 2, nonzero=True)
    Z = I.uniform_bits(rng, 64, n, 3)
    al = rng.normal(5, 4)
    be = rng.normal(5, 5)

    def F(t):
        _, _, s1, s2 = oracle.expval(n, G, A, Z, t)
        return -np.sum(al * s1 + be * s2 / 2)

    g = oracle.expval_grad(n, G, A, Z, th, al, be)
    fd = _fd(F, th)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-7
    # Linear loss sum_a w_a <Z_a>^: alpha = -w/s, beta = 0.
    w = rng.normal(5, 6)
    g2 = oracle.expval_grad(n, G, A, Z, th, -w / 64.0, None)
    fd2 = _fd(lambda t: float(np.dot(w, oracle.expval(n, G, A, Z, t)[0])), th)
    assert np.linalg.norm(g2 - fd2) / np.linalg.norm(fd2) < 1e-7


def test_grad_zero_at_theta_zero():
    p = I.tiny_local(seed=8, s=128)
    g = oracle.expval_grad(p.n, p.G, p.A, p.Z, np.zeros(p.m), np.ones(p.l), np.ones(p.l))
    assert np.all(g == 0.0)


def test_bitflip_grad_matches_central_differences():
    """Stochastic bitflip circuit (eq. expval_bitflip): the product-rule
    gradient against central differences of the product form."""
    rng = I.Rng(45)
    n = 9
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.5
    A = I.bernoulli_bits(rng, 12, n, 0.5, 2, nonzero=True)
    w = rng.normal(12, 3)
    g = oracle.bitflip_grad(n, G, A, th, w)
    fd = _fd(lambda t: float(np.dot(w, oracle.bitflip_expval(n, G, A, t))), th)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-8


def test_bitflip_model_is_the_ancilla_iqp_circuit():
    """Sec. 2.5: the bitflip circuit equals the IQP circuit on n + m qubits
    whose gate j also acts on its own ancilla n + j, observed on the first n
    qubits; its exact expectation (enumeration over all 2^(n+m) samples) is
    the product form."""
    rng = I.Rng(46)
    n, m = 4, 6
    gates = [list(np.nonzero(b)[0]) for b in (rng.uniform(m * n, 1).reshape(m, n) < 0.5)]
    gates = [g if g else [0] for g in gates]
    th = rng.normal(m, 2) * 0.7
    A = I.bernoulli_bits(rng, 10, n, 0.5, 3)
    G = I.pack_index_lists(gates, n)
    G_anc = I.pack_index_lists([g + [n + j] for j, g in enumerate(gates)], n + m)
    A_anc = I.pack_bits(np.concatenate([I.unpack_bits(A, n), np.zeros((10, m), np.uint8)], axis=1))
    exact = oracle.exact_expval(n + m, G_anc, A_anc, th)
    assert np.max(np.abs(exact - oracle.bitflip_expval(n, G, A, th))) < 1e-12


# ---------------------------------------------------------------------- MMD

def test_mmd_kernel_identity():
    """sum_a P_sigma(a) (<Z_a>_p - <Z_a>_q)^2 equals the Gaussian-kernel MMD^2
    sum_{x,y} (p-q)(x)(p-q)(y) exp(-|x-y|^2 / (2 sigma^2)) (eqs. mmd_loss and
    mmd_estimate) when observable bits are i.i.d. Bernoulli(p_sigma),
    p_sigma = (1 - exp(-1/(2 sigma^2)))/2; q is the statevector distribution
    and p the empirical data distribution."""
    rng = I.Rng(51)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.5
    X = I.prototype_data(rng, 40, n, 3, 0.1, 2)
    sigma2 = 1.7
    ps = I.p_sigma(sigma2)
    strings = all_strings(n)
    # Model: estimator over every z is exact; data: empirical distribution.
    _, terms, _ = oracle.mmd_loss(n, G, strings, strings, X, th, unbiased=False)
    abits = bits_of(strings, n)
    w = np.prod(np.where(abits == 1, ps, 1 - ps), axis=1)
    observable_form = float(np.dot(w, terms))

    q = oracle.statevector_probs(n, G, th)
    xs = np.arange(1 << n)
    idx = bits_of(X, n) @ (1 << np.arange(n))
    p = np.bincount(idx, minlength=1 << n) / X.shape[0]
    d = p - q
    ham = np.array([[bin(x ^ y).count("1") for y in xs] for x in xs])
    kernel_form = float(d @ np.exp(-ham / (2 * sigma2)) @ d)
    assert abs(observable_form - kernel_form) < 1e-12
    assert kernel_form > 1e-4  # non-trivial


def test_mmd_unbiased_terms_are_pair_means():
    """U-statistics: (S1^2 - S2)/(s(s-1)) is the mean of cos_i cos_k over i != k
    and (T^2 - N)/(N(N-1)) the mean of (-1)^{a.x}(-1)^{a.y} over x != y."""
    rng = I.Rng(52)
    n = 7
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.3
    A = I.bernoulli_bits(rng, 6, n, 0.3, 2, nonzero=True)
    Z = I.uniform_bits(rng, 9, n, 3)
    X = I.uniform_bits(rng, 7, n, 4)
    s, N, l = Z.shape[0], X.shape[0], A.shape[0]
    cos_each = np.stack([oracle.expval(n, G, A, Z[i:i + 1], th)[2] for i in range(s)], axis=1)
    sgn_each = np.stack([oracle.data_parity_sum(n, A, X[x:x + 1]) for x in range(N)], axis=1)
    want = []
    for a in range(l):
        uq = np.mean([cos_each[a, i] * cos_each[a, k] for i in range(s) for k in range(s) if i != k])
        up = np.mean([sgn_each[a, x] * sgn_each[a, y] for x in range(N) for y in range(N) if x != y])
        cross = 2 * sgn_each[a].mean() * cos_each[a].mean()
        want.append(up - cross + uq)
    loss, terms, _ = oracle.mmd_loss(n, G, A, Z, X, th, unbiased=True)
    assert np.max(np.abs(terms - np.array(want))) < 1e-13
    assert abs(loss - np.mean(want)) < 1e-13


@pytest.mark.parametrize("unbiased", [True, False])
def test_mmd_grad_matches_central_differences(unbiased):
    rng = I.Rng(53)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.3
    A = I.bernoulli_bits(rng, 8, n, 0.4, 2, nonzero=True)
    Z = I.uniform_bits(rng, 40, n, 3)
    X = I.prototype_data(rng, 30, n, 2, 0.1, 4)
    _, _, g = oracle.mmd_loss(n, G, A, Z, X, th, unbiased=unbiased, grad=True)
    fd = _fd(lambda t: oracle.mmd_loss(n, G, A, Z, X, t, unbiased=unbiased)[0], th)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-6


def test_mmd_unbiased_in_expectation_over_samples():
    """E_Z[U_q] = <Z_a>_q^2: average the U-statistic over many independent
    sample batches and compare with the exact value squared."""
    rng = I.Rng(54)
    n = 5
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.4
    A = I.bernoulli_bits(rng, 4, n, 0.5, 2, nonzero=True)
    exact = oracle.exact_expval(n, G, A, th)
    s, reps = 6, 3000
    Zall = I.uniform_bits(rng, s * reps, n, 3)
    _, _, S1, S2 = oracle.expval(n, G, np.repeat(A, 1, axis=0), Zall[:s], th)
    acc = np.zeros(A.shape[0])
    for r in range(reps):
        _, _, S1, S2 = oracle.expval(n, G, A, Zall[r * s:(r + 1) * s], th)
        acc += (S1 ** 2 - S2) / (s * (s - 1))
    est = acc / reps
    assert np.max(np.abs(est - exact ** 2)) < 0.03


# ---------------------------------------------------------- input recipes

def test_local_gates_order_matches_paper():
    gold = json.load(open(GOLDEN))["local_gates_n3"]["value"]
    assert I.local_gates(3) == gold
    assert np.array_equal(I.local_gates_packed(9), I.pack_index_lists(I.local_gates(9), 9))


def test_pack_roundtrip_and_padding():
    rng = I.Rng(61)
    for n in (1, 63, 64, 65, 130, 300):
        b = (rng.uniform(7 * n, 1).reshape(7, n) < 0.5).astype(np.uint8)
        w = I.pack_bits(b)
        assert w.shape[1] % 2 == 0
        assert np.array_equal(I.unpack_bits(w, n), b)
        assert np.array_equal(I.unpack_bits(w, w.shape[1] * 64)[:, n:], np.zeros((7, w.shape[1] * 64 - n)))


def test_random_k_body_distinct_qubits():
    rng = I.Rng(62)
    G = I.random_k_body(rng, 5000, 17, [1, 2, 3], 1)
    k = bits_of(G, 17).sum(axis=1)
    assert set(np.unique(k)) == {1, 2, 3}
    assert abs(np.mean(k) - 2.0) < 0.05


# ------------------------------------------------------------ API variants

def test_mmd_sqrt_loss_grad_matches_central_differences():
    """sqrt_loss (Sec. 3.3.1): the gradient of sqrt(MMD^2) by central
    differences of the square-rooted loss itself."""
    rng = I.Rng(55)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.3
    A = I.bernoulli_bits(rng, 8, n, 0.4, 2, nonzero=True)
    Z = I.uniform_bits(rng, 40, n, 3)
    X = I.prototype_data(rng, 30, n, 2, 0.1, 4)
    for unbiased in (True, False):
        L, g = oracle.mmd_loss_sqrt(n, G, A, Z, X, th, unbiased, grad=True)
        assert L > 0.05
        fd = _fd(lambda t: oracle.mmd_loss_sqrt(n, G, A, Z, X, t, unbiased)[0], th)
        assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-6


def _pauli_x_string(n, qubits):
    """Dense 2^n x 2^n matrix of prod_{q in qubits} X_q (basis index bit q =
    qubit q): it maps |x> to |x xor mask>."""
    mask = sum(1 << q for q in qubits)
    M = np.zeros((1 << n, 1 << n))
    for x in range(1 << n):
        M[x ^ mask, x] = 1.0
    return M


def test_shared_parameter_gates_match_matrix_exponential():
    """The paper's shared-parameter example on three qubits: gate 1 =
    exp(i theta_1 (X I X + X X X)), gate 2 = exp(i theta_2 X I I). The
    expanded generator list with per-generator parameters must reproduce the
    state exp(i H)|0> built by a dense matrix exponential of the summed
    generators, for every observable."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    gold = json.load(open(GOLDEN))["shared_parameter_example_n3"]["value"]
    n = 3
    gens, start = [], [0]
    for gate in gold:
        gens.extend(gate)
        start.append(len(gens))
    G = I.pack_index_lists(gens, n)
    th_p = np.array([0.37, -0.81])
    H = sum(th_p[p] * _pauli_x_string(n, g) for p, gate in enumerate(gold) for g in gate)
    psi = scipy_linalg.expm(1j * H)[:, 0]
    probs = np.abs(psi) ** 2
    A = all_strings(n)
    signs = (-1.0) ** (bits_of(A, n) @ bits_of(all_strings(n), n).T)
    want = signs @ probs
    got = oracle.exact_expval(n, G, A, oracle.expand_params(th_p, start))
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.max(np.abs(want - 1.0)) > 0.1  # not trivial


def test_shared_parameter_grad_matches_central_differences():
    """Chain rule through shared parameters: the gate gradient is the sum of
    its generators' gradients; checked by central differences in theta_p of
    the estimator evaluated with the expanded parameters."""
    rng = I.Rng(56)
    n = 7
    gens = [[0, 2], [0, 1, 2], [0], [3, 4], [5], [1, 6], [2, 3, 5]]
    start = [0, 2, 3, 5, 7]
    G = I.pack_index_lists(gens, n)
    th_p = rng.normal(4, 1) * 0.4
    A = I.bernoulli_bits(rng, 6, n, 0.4, 2, nonzero=True)
    Z = I.uniform_bits(rng, 64, n, 3)
    w = rng.normal(A.shape[0], 4)
    alpha = -w / Z.shape[0]
    g_gen = oracle.expval_grad(n, G, A, Z, oracle.expand_params(th_p, start), alpha)
    g_p = oracle.reduce_params(g_gen, start)
    fd = _fd(lambda t: float(np.dot(w, oracle.expval(n, G, A, Z, oracle.expand_params(t, start))[0])), th_p)
    assert np.linalg.norm(g_p - fd) / np.linalg.norm(fd) < 1e-7


def test_mmd_with_wires_is_kernel_mmd_of_the_marginal():
    """wires (Sec. 3.3.1): with observables and data on the wire qubits only,
    sum_a P_sigma(a) term_a over all a on the wires equals the Gaussian-kernel
    MMD^2 between the data and the circuit's marginal distribution on the
    wires (ancillas summed out of the statevector probabilities)."""
    rng = I.Rng(57)
    n, wires = 5, [0, 2, 3]
    nw = len(wires)
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.5
    Xw = I.prototype_data(rng, 40, nw, 2, 0.15, 2)
    sigma2 = 0.9
    ps = I.p_sigma(sigma2)
    Aw = all_strings(nw)
    A = oracle.embed_bits(Aw, nw, wires, n)
    X = oracle.embed_bits(Xw, nw, wires, n)
    _, terms, _ = oracle.mmd_loss(n, G, A, all_strings(n), X, th, unbiased=False)
    abits = bits_of(Aw, nw)
    wgt = np.prod(np.where(abits == 1, ps, 1 - ps), axis=1)
    observable_form = float(np.dot(wgt, terms))

    probs = oracle.statevector_probs(n, G, th)
    xs = np.arange(1 << n)
    wire_index = sum(((xs >> q) & 1) << k for k, q in enumerate(wires))
    q_marg = np.bincount(wire_index, weights=probs, minlength=1 << nw)
    idx = bits_of(Xw, nw) @ (1 << np.arange(nw))
    p_data = np.bincount(idx, minlength=1 << nw) / Xw.shape[0]
    d = p_data - q_marg
    ys = np.arange(1 << nw)
    ham = np.array([[bin(x ^ y).count("1") for y in ys] for x in ys])
    kernel_form = float(d @ np.exp(-ham / (2 * sigma2)) @ d)
    assert abs(observable_form - kernel_form) < 1e-12
    assert kernel_form > 1e-4


def test_embed_bits_places_each_wire():
    rng = I.Rng(58)
    n, wires = 130, [129, 0, 64, 63, 7]
    src = I.uniform_bits(rng, 9, len(wires), 1)
    out = oracle.embed_bits(src, len(wires), wires, n)
    want = np.zeros((9, n), np.uint8)
    want[:, wires] = I.unpack_bits(src, len(wires))
    assert np.array_equal(I.unpack_bits(out, n), want)
    assert np.array_equal(out, I.pack_bits(want))  # padding bits zero


def test_indep_estimates_are_independent_and_unbiased():
    """indep_estimates (Sec. 2.2): with one batch per observable, copies of the
    same observable get independent estimates whose spread matches the
    single-estimate variance Var(cos Phi)/s, each within 3 SE of the exact
    value; with a shared batch the copies would be identical."""
    rng = I.Rng(59)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.35
    a = I.bernoulli_bits(rng, 1, n, 0.5, 2, nonzero=True)
    copies, s = 400, 64
    A = np.repeat(a, copies, axis=0)
    Z = I.uniform_bits(rng, copies * s, n, 3)
    ev, se, _, _ = oracle.expval_indep(n, G, A, Z, th)
    exact = float(oracle.exact_expval(n, G, a, th)[0])
    # Var(cos Phi) over z ~ U{0,1}^n, exactly: E[cos^2] - E[cos]^2.
    allz = all_strings(n)
    _, _, s1, s2 = oracle.expval(n, G, a, allz, th)
    var = s2[0] / allz.shape[0] - (s1[0] / allz.shape[0]) ** 2
    spread = float(np.var(ev))
    assert abs(spread / (var / s) - 1.0) < 0.25  # chi-square with 399 dof: sd ~ 0.07
    assert abs(float(np.mean(ev)) - exact) < 4 * math.sqrt(var / s / copies)
    assert np.mean(np.abs(ev - exact) <= 3 * se) > 0.97
    ev_shared, _, _, _ = oracle.expval(n, G, A, Z[:s], th)
    assert np.all(ev_shared == ev_shared[0])


def test_indep_grad_matches_central_differences():
    rng = I.Rng(60)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.3
    A = I.bernoulli_bits(rng, 5, n, 0.4, 2, nonzero=True)
    s = 30
    Z = I.uniform_bits(rng, A.shape[0] * s, n, 3)
    w = rng.normal(A.shape[0], 4)
    g = oracle.expval_indep_grad(n, G, A, Z, th, -w / s)
    fd = _fd(lambda t: float(np.dot(w, oracle.expval_indep(n, G, A, Z, t)[0])), th)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-7


def test_mmd_indep_with_repeated_batch_equals_shared_batch():
    """indep_estimates with every observable given the same batch is the
    shared-batch estimator (loss, terms and gradient)."""
    rng = I.Rng(61)
    n = 6
    G = I.local_gates_packed(n)
    th = rng.normal(G.shape[0], 1) * 0.3
    A = I.bernoulli_bits(rng, 5, n, 0.4, 2, nonzero=True)
    Z = I.uniform_bits(rng, 33, n, 3)
    X = I.prototype_data(rng, 20, n, 2, 0.1, 4)
    for unbiased in (True, False):
        L0, t0, g0 = oracle.mmd_loss(n, G, A, Z, X, th, unbiased, grad=True)
        L1, t1, g1 = oracle.mmd_loss_ex(n, G, A, np.tile(Z, (A.shape[0], 1)), X, th, unbiased, indep=True,
                                        grad=True)
        assert abs(L0 - L1) < 1e-14 and np.max(np.abs(t0 - t1)) < 1e-14
        assert np.max(np.abs(g0 - g1)) < 1e-12


# ------------------------------------------------------------ low-order regrouping

def _low_order_problem(seed, n=11, m=70, l=23, s=97):
    """Random one- and two-body generators in random order, with repeated
    supports, plus observables and samples."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(m):
        if rng.random() < 0.3:
            gates.append([int(rng.integers(n))])
        else:
            q, r = sorted(int(x) for x in rng.choice(n, 2, replace=False))
            gates.append([q, r])
    gates += gates[:5]  # repeated supports add their angles
    theta = rng.normal(0.0, 0.4, len(gates))
    a = (rng.random((l, n)) < 0.4).astype(np.int64)
    z = rng.integers(0, 2, (s, n))
    return gates, theta, a, z


def _pair_coefficients(gates, theta, n):
    """d_q = sum of 2 theta over gates on {q}; C_qr = C_rq = sum of 2 theta
    over gates on {q, r}."""
    d, C = np.zeros(n), np.zeros((n, n))
    for g, t in zip(gates, theta):
        if len(g) == 1:
            d[g[0]] += 2 * t
        else:
            C[g[0], g[1]] += 2 * t
            C[g[1], g[0]] += 2 * t
    return d, C


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_low_order_regrouping_of_the_phase(seed):
    """For generators of weight <= 2 the phase of eq. expvalsample factors per
    qubit: [g.a odd] s_g = (a_q + a_r - 2 a_q a_r) s_q s_r for g = {q, r}, so
    Phi(a, z) = sum_{q in a} s_q (d_q + (C s)_q) - 2 sum_{q<r in a} C_qr s_q s_r
    with s = 1 - 2z. The oracle evaluates the phase gate by gate; the
    regrouped form here never forms a gate parity."""
    n = 11
    gates, theta, a, z = _low_order_problem(seed, n)
    d, C = _pair_coefficients(gates, theta, n)
    S = 1 - 2 * z
    lin = a @ (S * (d + S @ C)).T                        # [l, s]
    U = a[:, None, :] * S[None, :, :]                    # a_q s_q
    quad = 0.5 * np.einsum("lsq,qr,lsr->ls", U, C, U)    # sum_{q<r}
    phi = lin - 2 * quad
    ev, se, _, _ = oracle.expval(n, I.pack_index_lists(gates, n), I.pack_bits(a),
                                 I.pack_bits(z), theta)
    want = np.cos(phi).mean(axis=1)
    assert np.abs(ev - want).max() < 1e-12
    sd = np.cos(phi).std(axis=1, ddof=0) / math.sqrt(z.shape[0])
    assert np.abs(se - sd).max() < 1e-12


@pytest.mark.parametrize("seed", [4, 5])
def test_low_order_regrouping_of_the_gradient(seed):
    """The gradient of the regrouped phase: with V = sin(Phi)(alpha + beta cos Phi),
    a one-body gate on q gets 2 sum V a_q s_q and a pair gate on {q, r} gets
    2 sum V (a_q + a_r - 2 a_q a_r) s_q s_r; gates sharing a support share
    the value."""
    n = 11
    gates, theta, a, z = _low_order_problem(seed, n)
    rng = np.random.default_rng(seed + 100)
    alpha, beta = rng.normal(size=a.shape[0]), rng.normal(size=a.shape[0])
    d, C = _pair_coefficients(gates, theta, n)
    S = 1 - 2 * z
    U = a[:, None, :] * S[None, :, :]
    phi = a @ (S * (d + S @ C)).T - np.einsum("lsq,qr,lsr->ls", U, C, U)
    V = np.sin(phi) * (alpha[:, None] + beta[:, None] * np.cos(phi))
    K = a.T @ V                                          # [n, s]: sum_a V a_q
    M1 = (K * S.T) @ S                                   # sum V a_q s_q s_r
    Q = np.einsum("ls,lq,lr,sq,sr->qr", V, a, a, S, S)   # sum V a_q a_r s_q s_r
    M0 = (K * S.T).sum(axis=1)                           # sum V a_q s_q
    want = np.array([2 * M0[g[0]] if len(g) == 1 else
                     2 * (M1[g[0], g[1]] + M1[g[1], g[0]] - 2 * Q[g[0], g[1]])
                     for g in gates])
    got = oracle.expval_grad(n, I.pack_index_lists(gates, n), I.pack_bits(a),
                             I.pack_bits(z), theta, alpha, beta)
    assert np.abs(got - want).max() < 1e-10 * max(1.0, np.abs(want).max())
