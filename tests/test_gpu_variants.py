"""GPU parity of the API options around the estimator, through the C ABI:
on-device random bits (bit-exact with the seeded host generators), the
`wires` embedding and shared-parameter expansion / reduction (bit-exact with
the oracle), sqrt_loss, and independent per-observable sample batches
(indep_estimates) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_04776_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
GRAD_RTOL = 1e-4


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


def host(t):
    return t.cpu().numpy().view(np.uint64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ RNG

@pytest.mark.parametrize("n,rows", [(1, 1), (63, 5), (64, 7), (65, 3), (130, 257), (1000, 33)])
def test_device_uniform_bits_match_host_generator(api, n, rows):
    for seed, stream in ((0, 1000), (12345, 7), (2 ** 63 + 5, 2 ** 40 + 3)):
        got = host(api.uniform_bits(seed, stream, rows, n))
        want = I.uniform_bits(I.Rng(seed), rows, n, stream)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("n,rows", [(1, 3), (63, 5), (64, 2), (130, 300), (1000, 17)])
@pytest.mark.parametrize("p", [0.0, 0.003984, 0.05, 0.5, 1.0])
def test_device_bernoulli_bits_match_host_generator(api, n, rows, p):
    got = host(api.bernoulli_bits(77, 1001, rows, n, p))
    want = I.bernoulli_bits(I.Rng(77), rows, n, p, 1001)
    assert np.array_equal(got, want)


def test_training_with_device_rng_matches_host_draws(api):
    """The training loop with on-device draws sees the same samples and
    observables as with host draws, so the loss trajectory is identical."""
    from paper_2501_04776_gb300 import train
    p = I.mmd_training(seed=7, n=12, l=64, s=256, N=200)
    _, host_losses = train.adam_mmd(p, steps=4, lr=0.05)
    _, dev_losses = train.adam_mmd(p, steps=4, lr=0.05, device_rng=True)
    assert host_losses == dev_losses


# ----------------------------------------------------- wires, parameters

def test_embed_bits_matches_oracle(api):
    rng = I.Rng(3)
    n, wires = 200, [199, 0, 64, 63, 7, 128, 127]
    src = I.uniform_bits(rng, 301, len(wires), 1)
    got = host(api.embed_bits(dev(api, src), len(wires), wires, n))
    assert np.array_equal(got, oracle.embed_bits(src, len(wires), wires, n))


def test_expand_and_reduce_params_match_oracle(api):
    import torch
    rng = I.Rng(4)
    sizes = rng.integers(500, 4, 1) + 1
    start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m = int(start[-1])
    th_p = (0.3 * rng.normal(500, 2)).astype(np.float32)
    th_gen = api.expand_params(th_dev(th_p), start, m)
    assert np.array_equal(th_gen.cpu().numpy(), oracle.expand_params(th_p.astype(np.float64), start).astype(np.float32))
    g = rng.normal(m, 3)
    th = th_dev(th_p).requires_grad_(True)
    api.expand_params(th, start, m).backward(torch.from_numpy(g).float().cuda())
    # the reduction runs in FP64 over float32 upstream values
    want = oracle.reduce_params(g.astype(np.float32).astype(np.float64), start)
    assert np.max(np.abs(th.grad.double().cpu().numpy() - want.astype(np.float32))) <= 1e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "sparse_fp32"])
def test_shared_parameter_gates_autograd(api, prec):
    """Gates that share parameters: expand -> estimator -> sum_a w_a <Z_a>,
    backward through the estimator and the reduction, against the oracle's
    chain rule."""
    import torch
    rng = I.Rng(5)
    n, ngates = 90, 400
    sizes = rng.integers(ngates, 3, 6) + 1
    start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m = int(start[-1])
    G = I.random_k_body(rng, m, n, [1, 2, 3], 7)
    A = I.bernoulli_bits(rng, 150, n, 0.1, 8)
    Z = I.uniform_bits(rng, 700, n, 9)
    th_p = (0.2 * rng.normal(ngates, 10)).astype(np.float32)
    w = rng.normal(A.shape[0], 11)
    theta = th_dev(th_p).requires_grad_(True)
    ev, _ = api.expval(api.expand_params(theta, start, m), dev(api, G), dev(api, A), dev(api, Z), n, prec)
    (ev * torch.from_numpy(w).cuda()).sum().backward()
    thg = oracle.expand_params(th_p.astype(np.float64), start)
    want_ev = oracle.expval(n, G, A, Z, thg)[0]
    tol = 1e-4 if prec == "split_bf16" else TOL32
    assert np.max(np.abs(ev.detach().cpu().numpy() - want_ev)) <= tol
    want = oracle.reduce_params(oracle.expval_grad(n, G, A, Z, thg, -w / Z.shape[0]), start)
    assert rel_l2(theta.grad.double().cpu().numpy(), want) <= GRAD_RTOL


# -------------------------------------------------------------- sqrt_loss

@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "sparse_fp32"])
@pytest.mark.parametrize("unbiased", [True, False])
def test_mmd_sqrt_loss(api, prec, unbiased):
    p = I.mmd_training(seed=11, n=50, l=200, s=500, N=300)
    th = (p.theta * 20).astype(np.float32)
    loss, grad = api.mmd_loss_raw(p.n, th_dev(th), dev(api, p.G), dev(api, p.A), dev(api, p.Z), dev(api, p.X),
                                  prec, unbiased, with_grad=True, sqrt_loss=True)
    want_loss, want_grad = oracle.mmd_loss_sqrt(p.n, p.G, p.A, p.Z, p.X, th.astype(np.float64), unbiased, grad=True)
    assert want_loss > 0
    tol = 1e-4 if prec == "split_bf16" else TOL32
    assert abs(float(loss) - want_loss) <= tol
    assert rel_l2(grad.cpu().numpy(), want_grad) <= GRAD_RTOL


# -------------------------------------------------------- indep_estimates

def _indep_problem(seed, n, m, l, s, ks=(1, 2, 3), pa=0.1, scale=0.3):
    rng = I.Rng(seed)
    G = I.random_k_body(rng, m, n, list(ks), 1)
    theta = (scale * rng.normal(m, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, pa, 3)
    Z = I.uniform_bits(rng, l * s, n, 4)
    return G, theta, A, Z


@pytest.mark.parametrize("n,m,l,s", [(8, 36, 5, 1), (130, 1000, 37, 600), (70, 300, 9, 4100), (1000, 5000, 6, 1000)])
def test_indep_estimates_match_oracle(api, n, m, l, s):
    G, th, A, Z = _indep_problem(20 + n, n, m, l, s)
    if n == 8:
        G = I.local_gates_packed(8)
        th = (0.3 * I.Rng(1).normal(G.shape[0], 1)).astype(np.float32)
    ev, se = api.expval_indep_raw(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z))
    want_ev, want_se, _, _ = oracle.expval_indep(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev.cpu().numpy() - want_ev)) <= TOL32
    assert np.max(np.abs(se.cpu().numpy() - want_se)) <= TOL32
    w = I.Rng(5).normal(l, 1)
    g = api.expval_indep_grad(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), -np_t(w) / s)
    want = oracle.expval_indep_grad(n, G, A, Z, th.astype(np.float64), -w / s)
    assert rel_l2(g.cpu().numpy(), want) <= GRAD_RTOL


def np_t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def test_indep_estimates_with_wide_generators(api):
    """Generators of weight up to 9 (beyond the three listed support qubits:
    the kernel reads their support from G)."""
    n, m, l, s = 150, 400, 7, 900
    G, th, A, Z = _indep_problem(41, n, m, l, s, ks=(1, 2, 3))
    rng = I.Rng(42)
    wide = I.bernoulli_bits(rng, 60, n, 0.04, 5, nonzero=True)
    G = np.concatenate([G, wide])
    th = np.concatenate([th, (0.3 * rng.normal(60, 6)).astype(np.float32)])
    ev, se = api.expval_indep_raw(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z))
    want_ev, want_se, _, _ = oracle.expval_indep(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev.cpu().numpy() - want_ev)) <= TOL32
    g = api.expval_indep_grad(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), np_t(np.full(l, 1.0 / s)))
    want = oracle.expval_indep_grad(n, G, A, Z, th.astype(np.float64), np.full(l, 1.0 / s))
    assert rel_l2(g.cpu().numpy(), want) <= GRAD_RTOL


def test_indep_autograd_and_mmd(api):
    import torch
    n, m, l, s = 60, 500, 40, 300
    G, th, A, Z = _indep_problem(43, n, m, l, s)
    theta = th_dev(th).requires_grad_(True)
    ev, _ = api.expval_indep(theta, dev(api, G), dev(api, A), dev(api, Z), n)
    w = I.Rng(44).normal(l, 1)
    (ev * np_t(w)).sum().backward()
    want = oracle.expval_indep_grad(n, G, A, Z, th.astype(np.float64), -w / s)
    assert rel_l2(theta.grad.double().cpu().numpy(), want) <= GRAD_RTOL
    X = I.prototype_data(I.Rng(45), 200, n, 4, 0.1, 1)
    for unbiased in (True, False):
        for sq in (False, True):
            loss, grad = api.mmd_loss_raw(n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), dev(api, X),
                                          "split_bf16", unbiased, with_grad=True, sqrt_loss=sq, indep=True)
            wl, _, wg = oracle.mmd_loss_ex(n, G, A, Z, X, th.astype(np.float64), unbiased, sq, True, grad=True)
            assert abs(float(loss) - wl) <= TOL32
            assert rel_l2(grad.cpu().numpy(), wg) <= GRAD_RTOL


def test_indep_gradient_is_reproducible(api):
    n, m, l, s = 60, 500, 40, 300
    G, th, A, Z = _indep_problem(46, n, m, l, s)
    args = (n, th_dev(th), dev(api, G), dev(api, A), dev(api, Z), np_t(np.full(l, 0.01)))
    assert np.array_equal(api.expval_indep_grad(*args).cpu().numpy(), api.expval_indep_grad(*args).cpu().numpy())
