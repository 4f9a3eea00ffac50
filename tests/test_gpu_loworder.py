"""GPU parity of the low-order form (IQP_LOWORDER_FP32: generators of weight
<= 2, phases regrouped through the n x n pair-coefficient matrix) against the
FP64 oracle, through the C ABI: estimates, standard errors, gradients and the
MMD loss, on local gate sets, random one- and two-body sets with duplicate
generators, heavy observables, and the full-size training and million-gate
shapes (sampled observables); plus its device-side argument errors."""
import numpy as np
import pytest

import oracle
from paper_2501_04776_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5
GRAD_RTOL = 1e-4
LO = "loworder_fp32"


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2501_04776_gb300 import build
    build.build()
    from paper_2501_04776_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def dev(api, words):
    return api.to_device_bits(words)


def th_dev(theta):
    import torch
    return torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float32)).cuda()


def t64(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(api, n, G, A, Z, th, w):
    from paper_2501_04776_gb300 import _lib
    ev, se = api.expval_raw(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), LO)
    g = api.expval_grad(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), t64(-w / Z.shape[0]), None, LO)
    assert api.read_status() == _lib.OK
    return ev.cpu().numpy(), se.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("n,l,s,pa", [(12, 40, 300, 0.3), (50, 200, 700, 0.1), (130, 97, 2100, 0.05),
                                      (200, 30, 513, 0.45)])
def test_local_gates_match_oracle(api, n, l, s, pa):
    """All one- and two-body gates on n qubits (observable weights up to ~90,
    beyond the 64 whose pair coefficients are staged in shared memory)."""
    rng = I.Rng(70 + n)
    G = I.local_gates_packed(n)
    th = (0.2 * rng.normal(G.shape[0], 1) / np.sqrt(n)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, pa, 2)
    A[0] = 0  # a = 0
    Z = I.uniform_bits(rng, s, n, 3)
    w = rng.normal(l, 4)
    ev, se, g = run(api, n, G, A, Z, th, w)
    want_ev, want_se, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL
    assert np.max(np.abs(se - want_se)) <= TOL
    assert ev[0] == 1.0
    want = oracle.expval_grad(n, G, A, Z, th.astype(np.float64), -w / s)
    assert rel_l2(g, want) <= GRAD_RTOL


def test_random_one_and_two_body_with_duplicates(api):
    """Random generators of weight 1 or 2 with repeated supports (their
    coefficients add), zero generators, and ragged sizes."""
    rng = I.Rng(81)
    n, m, l, s = 77, 3000, 150, 1000
    G = I.random_k_body(rng, m, n, [1, 2], 1)
    G[::97] = 0  # generators with empty support never contribute
    G = np.concatenate([G, G[:300]])  # duplicates
    th = (0.1 * rng.normal(G.shape[0], 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, 0.08, 3)
    Z = I.uniform_bits(rng, s, n, 4)
    w = rng.normal(l, 5)
    ev, se, g = run(api, n, G, A, Z, th, w)
    want_ev, want_se, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL and np.max(np.abs(se - want_se)) <= TOL
    want = oracle.expval_grad(n, G, A, Z, th.astype(np.float64), -w / s)
    assert rel_l2(g, want) <= GRAD_RTOL
    assert np.all(g[::97][:m // 97] == 0.0)


def test_mmd_loss_and_autograd(api):
    import torch
    p = I.mmd_training(seed=11, n=50, l=200, s=500, N=300)
    th = (p.theta * 20).astype(np.float32)
    for unbiased in (True, False):
        for sq in (False, True):
            loss, grad = api.mmd_loss_raw(p.n, th_dev(th), dev(api, p.G), dev(api, p.A), dev(api, p.Z),
                                          dev(api, p.X), LO, unbiased, with_grad=True, sqrt_loss=sq)
            wl, _, wg = oracle.mmd_loss_ex(p.n, p.G, p.A, p.Z, p.X, th.astype(np.float64), unbiased, sq, grad=True)
            assert abs(float(loss) - wl) <= TOL
            assert rel_l2(grad.cpu().numpy(), wg) <= GRAD_RTOL
    theta = th_dev(th).requires_grad_(True)
    ev, _ = api.expval(theta, dev(api, p.G), dev(api, p.A), dev(api, p.Z), p.n, LO)
    (3.0 * ev.sum()).backward()
    want = oracle.expval_grad(p.n, p.G, p.A, p.Z, th.astype(np.float64), np.full(p.l, -3.0 / p.Z.shape[0]))
    assert rel_l2(theta.grad.double().cpu().numpy(), want) <= GRAD_RTOL


def test_heavy_observables_take_the_one_sample_form(api):
    """Observables of 100 to 707 qubits in one launch: supports of at most
    256 qubits run four samples per thread, larger ones one sample per thread,
    and the heaviest carry more generator pairs than one pair list holds (the
    list is rebuilt round by round). Weights 256 and 257 sit on the boundary.
    Estimates, gradient, and the MMD loss and gradient (Phi kept from the
    statistics pass) against the oracle; s = 701 leaves a ragged last word."""
    rng = I.Rng(95)
    n, m, s = 1200, 5000, 701
    G = I.random_k_body(rng, m, n, [1, 2], 1)
    A = np.concatenate([I.bernoulli_bits(rng, 2, n, pa, 2 + k) for k, pa in enumerate((0.1, 0.4, 0.35, 0.6))])
    edge = np.zeros((2, n), np.uint8)
    edge[0, :256] = 1
    edge[1, 3:260] = 1
    A = np.concatenate([A, I.pack_bits(edge)])
    weights = I.unpack_bits(A, n).sum(axis=1)
    assert weights.min() <= 256 < weights.max() and 256 in weights and 257 in weights
    Z = I.uniform_bits(rng, s, n, 9)
    X = I.uniform_bits(rng, 40, n, 10)
    th = (0.05 * rng.normal(m, 3)).astype(np.float32)
    w = rng.normal(A.shape[0], 4)
    ev, se, g = run(api, n, G, A, Z, th, w)
    want_ev, want_se, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL and np.max(np.abs(se - want_se)) <= TOL
    assert rel_l2(g, oracle.expval_grad(n, G, A, Z, th.astype(np.float64), -w / s)) <= GRAD_RTOL
    loss, grad = api.mmd_loss_raw(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), dev(api, X), LO, True,
                                  with_grad=True)
    wl, _, wg = oracle.mmd_loss_ex(n, G, A, Z, X, th.astype(np.float64), True, False, grad=True)
    assert abs(float(loss) - wl) <= TOL
    assert rel_l2(grad.cpu().numpy(), wg) <= GRAD_RTOL


def test_gradient_is_reproducible(api):
    p = I.mmd_training(seed=12, n=60, l=100, s=800, N=10)
    args = (p.n, th_dev(p.theta * 10), dev(api, p.G), dev(api, p.A), dev(api, p.Z), t64(np.full(p.l, 0.01)), None,
            LO)
    assert np.array_equal(api.expval_grad(*args).cpu().numpy(), api.expval_grad(*args).cpu().numpy())


def test_repeated_supports_are_reproducible(api):
    """Every support repeated 40 times (their coefficients add into one C or
    d entry): estimates and gradient are the same bit for bit on every call,
    and match the oracle."""
    rng = I.Rng(13)
    n, l, s = 64, 50, 700
    base = I.random_k_body(rng, 120, n, [1, 2], 1)
    G = np.concatenate([base] * 40)
    th = (0.02 * rng.normal(G.shape[0], 2)).astype(np.float32)
    A, Z = I.bernoulli_bits(rng, l, n, 0.2, 3), I.uniform_bits(rng, s, n, 4)
    w = rng.normal(l, 5)
    runs = [run(api, n, G, A, Z, th, w) for _ in range(3)]
    for ev, se, g in runs[1:]:
        assert np.array_equal(ev, runs[0][0]) and np.array_equal(se, runs[0][1]) and np.array_equal(g, runs[0][2])
    want_ev, want_se, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(runs[0][0] - want_ev)) <= TOL and np.max(np.abs(runs[0][1] - want_se)) <= TOL
    assert rel_l2(runs[0][2], oracle.expval_grad(n, G, A, Z, th.astype(np.float64), -w / s)) <= GRAD_RTOL


def _relevant_gates(n, G, A_sub):
    return np.nonzero(oracle.parity(n, A_sub, G).any(axis=0))[0]


def test_full_size_mmd_training_shape(api):
    """n=1000, m=500500, l=2000, s=5000, N=10000 on a 32-observable subsample."""
    p = I.mmd_training(n=1000, l=2000, s=5000, N=10_000)
    p.theta = (p.theta * 10).astype(np.float32)
    idx = np.unique(np.sort(I.Rng(51).integers(32, p.l, 1)))
    A = p.A[idx]
    J = _relevant_gates(p.n, p.G, A)
    loss, grad = api.mmd_loss_raw(p.n, th_dev(p.theta), dev(api, p.G), dev(api, A), dev(api, p.Z), dev(api, p.X),
                                  LO, True, with_grad=True)
    want_loss, _, wg = oracle.mmd_loss(p.n, p.G[J], A, p.Z, p.X, p.theta.astype(np.float64)[J], True, grad=True)
    want_grad = np.zeros(p.m)
    want_grad[J] = wg
    assert abs(float(loss) - want_loss) <= TOL
    assert rel_l2(grad.cpu().numpy(), want_grad) <= GRAD_RTOL


def test_full_size_million_gates(api):
    """n=5000, m=1e6 one- and two-body gates, 4096 observables, 16384 samples,
    sampled observables (the oracle restricted to their relevant gates)."""
    p = I.million_gates()
    ev, se = api.expval_raw(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z), LO)
    idx = np.unique(np.sort(I.Rng(41).integers(6, p.l, 1)))
    A = p.A[idx]
    J = _relevant_gates(p.n, p.G, A)
    th = p.theta.astype(np.float64)
    S1 = np.zeros(idx.size)
    S2 = np.zeros(idx.size)
    for i0 in range(0, p.s, 4096):
        _, _, s1, s2 = oracle.expval(p.n, p.G[J], A, p.Z[i0:i0 + 4096], th[J])
        S1 += s1
        S2 += s2
    mean = S1 / p.s
    assert np.max(np.abs(ev.cpu().numpy()[idx] - mean)) <= TOL
    alpha = np.zeros(p.l)
    alpha[idx] = I.Rng(42).normal(idx.size, 1) / p.s
    g = api.expval_grad(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z), t64(alpha), None, LO)
    want = np.zeros(p.m)
    for i0 in range(0, p.s, 4096):
        want[J] += oracle.expval_grad(p.n, p.G[J], A, p.Z[i0:i0 + 4096], th[J], alpha[idx])
    assert rel_l2(g.cpu().numpy(), want) <= GRAD_RTOL


def test_device_errors_for_heavy_generators_and_observables(api):
    from paper_2501_04776_gb300 import _lib
    rng = I.Rng(90)
    n = 40
    G = I.random_k_body(rng, 50, n, [1, 2, 3], 1)  # some generators of weight 3
    A = I.bernoulli_bits(rng, 8, n, 0.2, 2)
    Z = I.uniform_bits(rng, 64, n, 3)
    api.expval_raw(n, th_dev(np.zeros(50)), dev(api, G), dev(api, A), dev(api, Z), LO)
    assert api.read_status() == _lib.ERR_ARG
    n = 2000
    G = I.local_gates_packed(60)
    G = np.concatenate([G, np.zeros((G.shape[0], I.words_per_row(n) - G.shape[1]), np.uint64)], axis=1)
    A = np.full((2, I.words_per_row(n)), np.uint64(0xFFFFFFFFFFFFFFFF))
    A[:, -2:] = 0  # 1920 qubits set in each observable
    Z = I.uniform_bits(rng, 64, n, 4)
    api.expval_raw(n, th_dev(np.zeros(G.shape[0])), dev(api, G), dev(api, A), dev(api, Z), LO)
    assert api.read_status() == _lib.ERR_UNSUPPORTED
    assert api.read_status() == _lib.OK  # cleared


@pytest.mark.parametrize("lo_tc", ["0", "1"])
def test_pair_contraction_forms_match_oracle(lo_tc):
    """Both forms of the pair contractions M = C S and H = (s o V) S^T: on the
    tensor cores (split BF16, the default) and as sign-flip FP32 additions
    over the pairs that carry a generator (IQP_LO_TC=0), on a ragged shape
    (n = 300: 300 rows in 256-row tiles, s = 1500), in a fresh process."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, numpy as np, torch, oracle
from paper_2501_04776_gb300 import api, inputs as I
rng = I.Rng(17)
n, l, s = 300, 120, 1500
G = I.local_gates_packed(n)
th = (0.02 * rng.normal(G.shape[0], 1)).astype(np.float32)
A = I.bernoulli_bits(rng, l, n, 0.03, 2); Z = I.uniform_bits(rng, s, n, 3)
w = rng.normal(l, 4)
d = api.to_device_bits
t = torch.from_numpy(th).cuda()
ev, se = api.expval_raw(n, t, d(G), d(A), d(Z), "loworder_fp32")
g = api.expval_grad(n, t, d(G), d(A), d(Z), torch.from_numpy(-w / s).cuda(), None, "loworder_fp32")
wev, wse, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
wg = oracle.expval_grad(n, G, A, Z, th.astype(np.float64), -w / s, None)
print(json.dumps({"ev": float(np.max(np.abs(ev.cpu().numpy() - wev))), "se": float(np.max(np.abs(se.cpu().numpy() - wse))),
                  "g": float(np.linalg.norm(g.cpu().numpy() - wg) / np.linalg.norm(wg)), "status": api.read_status()}))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, IQP_LO_TC=lo_tc, PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["status"] == 0
    assert r["ev"] <= TOL and r["se"] <= TOL and r["g"] <= GRAD_RTOL
