"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on
identical seeded inputs.

Bars: parities bit-exact; expectation values, standard errors and losses
within 1e-5 (FP32 form) / 1e-4 (split-BF16 form) absolute; gradients within
1e-4 relative L2. Shapes span several tiles with ragged tails; the full-size
cases run the exact launch configuration bench.py times and compare sampled
observables, which the oracle computes one by one.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2501_04776_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-4, "sparse_fp32": 1e-5, "loworder_fp32": 1e-5}
GRAD_RTOL = 1e-4
PRECS = ["fp32", "split_bf16", "sparse_fp32"]


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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_expval(api, p, prec, Z=None):
    Z = p.Z if Z is None else Z
    ev, se = api.expval_raw(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, Z), prec)
    return ev.cpu().numpy(), se.cpu().numpy()


def gpu_grad(api, p, alpha, beta, prec):
    import torch
    al = torch.from_numpy(np.asarray(alpha, dtype=np.float64)).cuda()
    be = None if beta is None else torch.from_numpy(np.asarray(beta, dtype=np.float64)).cuda()
    g = api.expval_grad(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z), al, be, prec)
    return g.cpu().numpy()


def ragged_problem(seed=7, n=130, m=1000, l=300, s=600, ks=(1, 2, 3), pa=0.1, scale=0.3):
    rng = I.Rng(seed)
    G = I.random_k_body(rng, m, n, list(ks), 1)
    theta = (scale * rng.normal(m, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, pa, 3)
    Z = I.uniform_bits(rng, s, n, 4)
    return I.Problem(f"ragged-n{n}-m{m}-l{l}-s{s}", n, G, A, Z, theta)


# ------------------------------------------------------------------ parity

@pytest.mark.parametrize("n,m,rows", [(1, 1, 1), (63, 65, 33), (130, 300, 257), (300, 1000, 70), (5000, 513, 40)])
def test_parity_bit_exact(api, n, m, rows):
    rng = I.Rng(100 + n)
    R = I.bernoulli_bits(rng, rows, n, 0.5, 1)
    G = I.random_k_body(rng, m, n, [1, 2, 3], 2) if n >= 3 else I.bernoulli_bits(rng, m, n, 0.5, 2)
    P = api.parity(n, dev(api, R), dev(api, G)).cpu().numpy().view(np.uint64)
    want = oracle.parity(n, R, G)
    got = I.unpack_bits(P, P.shape[1] * 64)
    assert np.array_equal(got[:, :m], want)
    assert not got[:, m:].any()  # padding bits are zero


@pytest.mark.parametrize("n,m,rows,dense", [(1, 1, 1, False), (63, 65, 33, False), (130, 300, 257, False),
                                            (300, 1000, 700, False), (5000, 513, 40, False), (777, 300, 129, True),
                                            (200, 1100, 2100, False), (1000, 1537, 1025, False)])
def test_parity_gather_bit_exact(api, n, m, rows, dense):
    rng = I.Rng(300 + n)
    R = I.bernoulli_bits(rng, rows, n, 0.5, 1)
    if dense or n < 3:
        G = I.bernoulli_bits(rng, m, n, 0.5, 2)
    else:
        G = I.random_k_body(rng, m, n, [1, 2, 3], 2)
    P, PT = api.parity_gather(n, dev(api, R), dev(api, G))
    P = P.cpu().numpy().view(np.uint64)
    PT = PT.cpu().numpy().view(np.uint64)
    want = oracle.parity(n, R, G)
    gotP = I.unpack_bits(P, P.shape[1] * 64)
    gotT = I.unpack_bits(PT, PT.shape[1] * 64)
    assert np.array_equal(gotP[:, :m], want) and not gotP[:, m:].any()
    assert np.array_equal(gotT[:, :rows], want.T) and not gotT[:, rows:].any()


def test_parity_dense_generators_bit_exact(api):
    rng = I.Rng(5)
    n, m, rows = 777, 300, 129
    R = I.bernoulli_bits(rng, rows, n, 0.5, 1)
    G = I.bernoulli_bits(rng, m, n, 0.5, 2)
    P = api.parity(n, dev(api, R), dev(api, G)).cpu().numpy().view(np.uint64)
    assert np.array_equal(I.unpack_bits(P, m), oracle.parity(n, R, G))


@pytest.mark.parametrize("n,l,N", [(8, 5, 3), (300, 70, 1000), (1000, 33, 2049)])
def test_parity_sum_exact(api, n, l, N):
    rng = I.Rng(200 + n)
    A = I.bernoulli_bits(rng, l, n, 0.2, 1)
    X = I.uniform_bits(rng, N, n, 2)
    T = api.parity_sum(n, dev(api, A), dev(api, X)).cpu().numpy()
    assert np.array_equal(T, oracle.data_parity_sum(n, A, X))


# -------------------------------------------------------------- estimator

@pytest.mark.parametrize("prec", PRECS)
def test_expval_local_n8(api, prec):
    """n=8, all one- and two-body gates, 64 observables, 1024 samples."""
    p = I.tiny_local(seed=1)
    ev, se = gpu_expval(api, p, prec)
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL[prec]
    assert np.max(np.abs(se - want_se)) <= TOL[prec]
    # Over all 2^8 sample strings the estimate is the exact expectation value,
    # which the oracle pins to a statevector.
    allz = I.pack_bits(np.array([[(z >> q) & 1 for q in range(8)] for z in range(256)]))
    ev_all, _ = gpu_expval(api, p, prec, Z=allz)
    exact = oracle.statevector_expval(p.n, p.G, p.A, p.theta.astype(np.float64))
    assert np.max(np.abs(ev_all - exact)) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_expval_ragged_tiles(api, prec):
    p = ragged_problem()
    ev, se = gpu_expval(api, p, prec)
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL[prec]
    assert np.max(np.abs(se - want_se)) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS + ["loworder_fp32"])
def test_expval_degenerate_cases(api, prec):
    rng = I.Rng(9)
    n = 70
    G = I.random_k_body(rng, 50, n, [1, 2], 1)
    theta = (0.4 * rng.normal(50, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, 5, n, 0.3, 3)
    A[0] = 0                      # a = 0: exactly 1
    Z = I.uniform_bits(rng, 1, n, 4)  # one sample: SE = 0, expval = cos Phi
    p = I.Problem("one-sample", n, G, A, Z, theta)
    ev, se = gpu_expval(api, p, prec)
    want, _, _, _ = oracle.expval(n, G, A, Z, theta.astype(np.float64))
    assert ev[0] == 1.0 and np.all(se == 0.0)
    assert np.max(np.abs(ev - want)) <= TOL[prec]
    # theta = 0: every estimate is exactly 1 with zero error.
    p0 = I.Problem("zero", n, G, A, I.uniform_bits(rng, 300, n, 5), np.zeros(50, np.float32))
    ev0, se0 = gpu_expval(api, p0, prec)
    assert np.all(ev0 == 1.0) and np.all(se0 == 0.0)
    # One gate, one qubit, one observable.
    p1 = I.Problem("single", 1, I.pack_index_lists([[0]], 1), I.pack_index_lists([[0]], 1),
                   I.uniform_bits(rng, 7, 1, 6), np.array([0.3], np.float32))
    ev1, se1 = gpu_expval(api, p1, prec)
    assert abs(ev1[0] - math.cos(2 * float(np.float32(0.3)))) <= TOL[prec]


# --------------------------------------------------------------- gradient

@pytest.mark.parametrize("prec", PRECS)
def test_grad_vs_oracle(api, prec):
    p = ragged_problem(seed=8, l=260, s=520)
    rng = I.Rng(3)
    alpha = rng.normal(p.l, 1) / p.s
    beta = rng.normal(p.l, 2) / p.s
    for b in (None, beta):
        g = gpu_grad(api, p, alpha, b, prec)
        want = oracle.expval_grad(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64), alpha, b)
        assert rel_l2(g, want) <= GRAD_RTOL


@pytest.mark.parametrize("prec", PRECS)
def test_autograd_linear_loss(api, prec):
    import torch
    p = ragged_problem(seed=10, l=140, s=300, m=700)
    w = I.Rng(4).normal(p.l, 1)
    theta = th_dev(p.theta).requires_grad_(True)
    ev, se = api.expval(theta, dev(api, p.G), dev(api, p.A), dev(api, p.Z), p.n, prec)
    loss = (ev * torch.from_numpy(w).cuda()).sum()
    loss.backward()
    want = oracle.expval_grad(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64), -w / p.s, None)
    assert theta.grad.dtype == torch.float32
    assert rel_l2(theta.grad.double().cpu().numpy(), want) <= GRAD_RTOL
    assert not se.requires_grad


@pytest.mark.parametrize("prec", ["split_bf16", "sparse_fp32", "loworder_fp32"])
def test_kept_phase_gives_the_recomputed_results_bit_for_bit(api, prec):
    """iqp_expval_keep_phi returns iqp_expval's estimates and
    iqp_expval_grad_from_phi iqp_expval_grad's gradient, bit for bit (W is
    formed from the kept Phi with the recompute's arithmetic), for a loss
    with a beta term; autograd with and without keep_phi agrees the same way;
    both match the oracle."""
    import torch
    if prec == "loworder_fp32":
        rng = I.Rng(31)
        n, l, s = 40, 70, 333
        G = I.local_gates_packed(n)
        th = (0.3 * rng.normal(G.shape[0], 1) / np.sqrt(n)).astype(np.float32)
        A, Z = I.bernoulli_bits(rng, l, n, 0.2, 2), I.uniform_bits(rng, s, n, 3)
    else:
        p = ragged_problem(seed=13, l=140, s=333, m=700)
        n, G, A, Z, th, l, s = p.n, p.G, p.A, p.Z, p.theta.astype(np.float32), p.l, p.s
    Gd, Ad, Zd, thd = dev(api, G), dev(api, A), dev(api, Z), th_dev(th)
    ev0, se0 = api.expval_raw(n, thd, Gd, Ad, Zd, prec)
    ev1, se1, phi = api.expval_keep_phi_raw(n, thd, Gd, Ad, Zd, prec)
    assert torch.equal(ev0, ev1) and torch.equal(se0, se1)
    rng = I.Rng(6)
    alpha = torch.from_numpy(rng.normal(l, 1) / s).cuda()
    beta = torch.from_numpy(rng.normal(l, 2) / s).cuda()
    g0 = api.expval_grad(n, thd, Gd, Ad, Zd, alpha, beta, prec)
    g1 = api.expval_grad_from_phi(n, thd, Gd, Ad, Zd, phi, alpha, beta, prec)
    assert torch.equal(g0, g1)
    # a wider row stride changes nothing
    ev2, se2, phi2 = api.expval_keep_phi_raw(n, thd, Gd, Ad, Zd, prec, ld=api.phi_ld(s) + 128)
    assert torch.equal(ev0, ev2) and torch.equal(se0, se2)
    assert torch.equal(g0, api.expval_grad_from_phi(n, thd, Gd, Ad, Zd, phi2, alpha, beta, prec))
    want = oracle.expval_grad(n, G, A, Z, th.astype(np.float64), alpha.cpu().numpy(), beta.cpu().numpy())
    assert rel_l2(g1.cpu().numpy(), want) <= GRAD_RTOL
    want_ev, _, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
    assert np.max(np.abs(ev1.cpu().numpy() - want_ev)) <= TOL[prec]
    w = torch.from_numpy(rng.normal(l, 3)).cuda()
    grads = []
    for keep in (True, False):
        theta = th_dev(th).requires_grad_(True)
        ev, _ = api.expval(theta, Gd, Ad, Zd, n, prec, keep_phi=keep)
        ((ev * w).sum() + (ev * ev).sum()).backward()
        grads.append(theta.grad)
    assert torch.equal(grads[0], grads[1])


@pytest.mark.parametrize("prec", PRECS)
def test_grad_central_differences_on_gpu(api, prec):
    """Directional derivative of the GPU estimator by central differences of
    the GPU forward (Richardson-extrapolated, so the O(h^2) term cancels),
    against the GPU gradient."""
    p = ragged_problem(seed=12, n=40, m=200, l=64, s=512, scale=0.5)
    w = I.Rng(5).normal(p.l, 1)
    g = gpu_grad(api, p, -w / p.s, None, prec)
    v = g / np.linalg.norm(g)  # steepest direction: g.v = |g|

    def F(th):
        q = I.Problem("fd", p.n, p.G, p.A, p.Z, th.astype(np.float32))
        return float(np.dot(w, gpu_expval(api, q, prec)[0]))

    th = p.theta.astype(np.float64)

    def D(h):
        return (F(th + h * v) - F(th - h * v)) / (2 * h)

    h = 2e-2
    fd = (4 * D(h / 2) - D(h)) / 3
    gv = float(np.dot(g, v))
    assert abs(gv) > 0.5
    assert abs(fd - gv) <= 1e-2 * abs(gv)


# -------------------------------------------------------------------- MMD

def mmd_problem(seed=11, n=50, l=200, s=500, N=300):
    p = I.mmd_training(seed=seed, n=n, l=l, s=s, N=N)
    p.theta = (p.theta * 20).astype(np.float32)  # move away from theta ~ 0
    return p


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("unbiased", [True, False])
def test_mmd_loss_and_grad(api, prec, unbiased):
    p = mmd_problem()
    args = (p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z), dev(api, p.X), prec, unbiased)
    loss_only, _ = api.mmd_loss_raw(*args, with_grad=False)
    loss, grad = api.mmd_loss_raw(*args, with_grad=True)
    want_loss, _, want_grad = oracle.mmd_loss(p.n, p.G, p.A, p.Z, p.X, p.theta.astype(np.float64), unbiased,
                                              grad=True)
    assert abs(float(loss_only) - want_loss) <= TOL[prec]
    assert abs(float(loss) - want_loss) <= TOL[prec]
    assert rel_l2(grad.cpu().numpy(), want_grad) <= GRAD_RTOL


def test_mmd_autograd(api):
    import torch
    p = mmd_problem(seed=13, l=120, s=300, N=200)
    theta = th_dev(p.theta).requires_grad_(True)
    loss = api.mmd_loss(theta, dev(api, p.G), dev(api, p.A), dev(api, p.Z), dev(api, p.X), p.n, "split_bf16")
    (3.0 * loss).backward()
    _, _, want = oracle.mmd_loss(p.n, p.G, p.A, p.Z, p.X, p.theta.astype(np.float64), True, grad=True)
    assert rel_l2(theta.grad.double().cpu().numpy(), 3.0 * want) <= GRAD_RTOL


# ------------------------------------------------------- full-size sampled

def _sampled_forward_check(api, p, prec, nsample, seed):
    ev, se = gpu_expval(api, p, prec)
    idx = np.sort(I.Rng(seed).integers(nsample, p.l, 1))
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A[idx], p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev[idx] - want_ev)) <= TOL[prec]
    assert np.max(np.abs(se[idx] - want_se)) <= TOL[prec]
    assert np.all(np.isfinite(ev)) and np.all(np.abs(ev) <= 1.0 + 1e-6)


def _sampled_grad_check(api, p, prec, nsample, seed):
    """Gradient at full size with alpha nonzero on a sample of observables:
    the others contribute exactly zero, so the oracle needs only the sample."""
    idx = np.sort(I.Rng(seed).integers(nsample, p.l, 1))
    idx = np.unique(idx)
    alpha = np.zeros(p.l)
    alpha[idx] = I.Rng(seed + 1).normal(idx.size, 1) / p.s
    g = gpu_grad(api, p, alpha, None, prec)
    want = oracle.expval_grad(p.n, p.G, p.A[idx], p.Z, p.theta.astype(np.float64), alpha[idx], None)
    assert rel_l2(g, want) <= GRAD_RTOL


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_random_gates_n1000(api, prec):
    """10000 observables x 10000 samples x 100000 gates, n = 1000 (the
    benchmark workload), sampled observables."""
    p = I.random_gates(n=1000)
    _sampled_forward_check(api, p, prec, 16, 21)
    _sampled_grad_check(api, p, prec, 8, 22)


def test_full_size_local_n300(api):
    """n=300, all 45150 one- and two-body gates, 1000 observables, 10000 samples."""
    p = I.local300()
    for prec in PRECS:
        _sampled_forward_check(api, p, prec, 12, 23)
    _sampled_grad_check(api, p, "split_bf16", 6, 24)


# ------------------------------------------------------------ robustness

def test_deterministic_repeat(api):
    p = ragged_problem(seed=14)
    for prec in PRECS:
        a = gpu_expval(api, p, prec)
        b = gpu_expval(api, p, prec)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        alpha = np.full(p.l, 1.0 / p.s)
        assert np.array_equal(gpu_grad(api, p, alpha, None, prec), gpu_grad(api, p, alpha, None, prec))


def test_bounded_wait_times_out_and_context_survives(api):
    import torch
    from paper_2501_04776_gb300 import _lib
    lib = _lib.load()
    ws = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.iqp_read_status(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st) == _lib.OK
    assert lib.iqp_selftest_timeout(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 0.2, st) == _lib.OK
    assert lib.iqp_read_status(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st) == _lib.ERR_TIMEOUT
    assert lib.iqp_read_status(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st) == _lib.OK  # cleared
    p = I.tiny_local(seed=2, s=256)
    ev, _ = gpu_expval(api, p, "split_bf16")
    want, _, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev - want)) <= TOL["split_bf16"]
    assert api.read_status() == _lib.OK


def test_workspace_too_small_is_rejected_and_the_split_scratch_is_optional(api):
    import torch
    from paper_2501_04776_gb300 import _lib
    lib = _lib.load()
    # 1000 gates (16 operand stages: a tile can split into 4 gate ranges),
    # 2 x 3 pair tiles, all of them in the last round
    rng = I.Rng(13)
    n_, m_, l_, s_ = 130, 1000, 260, 520
    Gb = I.random_k_body(rng, m_, n_, [1, 2, 3], 1)
    p = I.Problem("ragged-n130-m1000-l260-s520", n_, Gb, I.bernoulli_bits(rng, l_, n_, 0.1, 3),
                  I.uniform_bits(rng, s_, n_, 4), (0.3 * rng.normal(m_, 2)).astype(np.float32))
    G, A, Z = dev(api, p.G), dev(api, p.A), dev(api, p.Z)
    th = th_dev(p.theta)
    need = lib.iqp_workspace_bytes(_lib.OP_EXPVAL, p.n, p.m, p.l, p.s, 0, _lib.SPLIT_BF16)
    ws = torch.zeros(need, dtype=torch.uint8, device="cuda")
    out = torch.zeros(p.l, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    # The end of the split-BF16 workspace is optional: the split-tile scratch
    # (160 partial accumulators of 128 x 256 FP32 and 160 counters, rounded
    # to 256 bytes), the running sums of the two-sample-tile phase (160 CTAs
    # x 2 x 128 x 256 FP32) and the scratch of its balanced last round (640
    # such accumulators and 160 counters). Anything shorter than the rest is
    # rejected.
    rnd = lambda b: -(-b // 256) * 256
    optional = rnd(160 * 128 * 256 * 4 + 160 * 4) + 160 * 2 * 128 * 256 * 4 + rnd(640 * 128 * 256 * 4 + 160 * 4)

    def call(nbytes, res):
        return lib.iqp_expval(p.n, P(G.data_ptr()), p.m, G.shape[1], P(A.data_ptr()), p.l, A.shape[1],
                              P(Z.data_ptr()), p.s, Z.shape[1], P(th.data_ptr()), _lib.SPLIT_BF16,
                              P(res.data_ptr()), None, P(ws.data_ptr()), nbytes, None)

    assert call(need - optional - 256, out) == _lib.ERR_WORKSPACE
    # Without the optional part every phase tile runs whole (with it, this
    # problem runs as split parts only): the same estimates within the
    # split-BF16 tolerance.
    full = torch.zeros(p.l, dtype=torch.float64, device="cuda")
    assert call(need, full) == _lib.OK
    assert call(need - optional, out) == _lib.OK
    torch.cuda.synchronize()
    assert api.read_status() == _lib.OK
    want, _, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - want)) <= TOL["split_bf16"]
    assert np.max(np.abs(full.cpu().numpy() - want)) <= TOL["split_bf16"]


def test_launch_counter_counts_kernels(api):
    before = api.launch_count()
    p = I.tiny_local(seed=4, s=128)
    gpu_expval(api, p, "split_bf16")
    assert api.launch_count() - before >= 4  # parity x2, theta split, phase, finalize


# ------------------------------------------------ remaining workload shapes

def _relevant_gates(n, G, A_sub):
    """Gates that anticommute with at least one of the sampled observables.
    Every other gate has P_A = 0 on all of them, so it adds exactly zero to
    their phases and its gradient entry is exactly zero: the oracle can skip it."""
    return np.nonzero(oracle.parity(n, A_sub, G).any(axis=0))[0]


def _oracle_expval_chunked(n, G, A, Z, th, chunk=4096):
    """Oracle estimate over all samples, computed on sample chunks (bounded
    host memory); S1 and S2 are exact sums, so the mean and the population
    variance follow directly."""
    S1 = np.zeros(A.shape[0])
    S2 = np.zeros(A.shape[0])
    for i0 in range(0, Z.shape[0], chunk):
        _, _, s1, s2 = oracle.expval(n, G, A, Z[i0:i0 + chunk], th)
        S1 += s1
        S2 += s2
    s = Z.shape[0]
    mean = S1 / s
    var = np.maximum(S2 / s - mean ** 2, 0.0)
    return mean, np.sqrt(var / s)


def _oracle_grad_chunked(n, G, A, Z, th, alpha, chunk=4096):
    g = np.zeros(G.shape[0])
    for i0 in range(0, Z.shape[0], chunk):
        g += oracle.expval_grad(n, G, A, Z[i0:i0 + chunk], th, alpha, None)
    return g


def _sampled_big_check(api, p, seed, nsample, prec="split_bf16"):
    ev, se = gpu_expval(api, p, prec)
    idx = np.unique(np.sort(I.Rng(seed).integers(nsample, p.l, 1)))
    A = p.A[idx]
    J = _relevant_gates(p.n, p.G, A)
    G, th = p.G[J], p.theta.astype(np.float64)[J]
    want_ev, want_se = _oracle_expval_chunked(p.n, G, A, p.Z, th)
    assert np.max(np.abs(ev[idx] - want_ev)) <= TOL[prec]
    assert np.max(np.abs(se[idx] - want_se)) <= TOL[prec]
    alpha = np.zeros(p.l)
    alpha[idx] = I.Rng(seed + 1).normal(idx.size, 1) / p.s
    g = gpu_grad(api, p, alpha, None, prec)
    want = np.zeros(p.m)
    want[J] = _oracle_grad_chunked(p.n, G, A, p.Z, th, alpha[idx])
    assert rel_l2(g, want) <= GRAD_RTOL
    outside = np.ones(p.m, bool)
    outside[J] = False
    assert np.all(g[outside] == 0.0)


@pytest.mark.parametrize("n", [100, 5000])
def test_full_size_random_gates_other_widths(api, n):
    """10000 observables x 10000 samples x 100000 gates at n = 100 and 5000
    (split-BF16), sampled observables."""
    _sampled_big_check(api, I.random_gates(n=n), 31 + n, 8)


@pytest.mark.parametrize("prec", ["split_bf16", "sparse_fp32"])
def test_full_size_million_gates(api, prec):
    """n=5000, m=1e6 random one- and two-body gates, 4096 observables, 16384
    samples (bit-packed operands only), sampled observables."""
    _sampled_big_check(api, I.million_gates(), 41, 6, prec)


@pytest.mark.parametrize("prec", ["split_bf16", "sparse_fp32"])
def test_full_size_mmd_training_shapes(api, prec):
    """MMD loss + gradient with the training workload's full m = 500500, n =
    1000, s = 5000, N = 10000, on a 32-observable subsample (the loss is a
    mean over observables, so a subsample is itself a valid MMD estimate)."""
    p = I.mmd_training(n=1000, l=2000, s=5000, N=10_000)
    p.theta = (p.theta * 10).astype(np.float32)
    idx = np.unique(np.sort(I.Rng(51).integers(32, p.l, 1)))
    A = p.A[idx]
    J = _relevant_gates(p.n, p.G, A)
    for unbiased in (True, False):
        loss, grad = api.mmd_loss_raw(p.n, th_dev(p.theta), dev(api, p.G), dev(api, A), dev(api, p.Z),
                                      dev(api, p.X), prec, unbiased, with_grad=True)
        want_loss, _, wg = oracle.mmd_loss(p.n, p.G[J], A, p.Z, p.X, p.theta.astype(np.float64)[J], unbiased,
                                           grad=True)
        want_grad = np.zeros(p.m)
        want_grad[J] = wg
        assert abs(float(loss) - want_loss) <= TOL[prec]
        assert rel_l2(grad.cpu().numpy(), want_grad) <= GRAD_RTOL


def test_adam_on_mmd_loss_converges(api):
    """The training loop (fresh samples and observables every step, Adam)
    drives the MMD^2 loss of a small circuit towards the data."""
    from paper_2501_04776_gb300 import train
    p = I.mmd_training(seed=7, n=10, l=256, s=512, N=500)
    _, losses = train.adam_mmd(p, steps=60, lr=0.05)
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.3 * np.mean(losses[:5])


@pytest.mark.parametrize("pairs,split,tmem,gpair", [("0", "1", "1", "1"), ("2", "0", "1", "1"), ("0", "0", "1", "1"),
                                                   ("2", "1", "0", "1"), ("2", "1", "1", "0"), ("2", "0", "0", "0")])
def test_other_tensor_kernel_forms_match_oracle(pairs, split, tmem, gpair):
    """The tensor-core kernel forms the defaults do not use: one-CTA kernels
    (IQP_CTA_PAIRS=0), whole phase tiles without the split last round
    (IQP_SPLIT_TAIL=0; this small problem is all last round, so with the
    default every tile is split along the gates), the pair phase kernel with
    its A operand in shared memory instead of TMEM (IQP_PHASE_TMEM=0), and
    the single-CTA gradient contraction in place of the CTA-pair one
    (IQP_GRAD_PAIR=0), on the ragged problem, in a fresh process."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, numpy as np, torch, oracle
from paper_2501_04776_gb300 import api, inputs as I
rng = I.Rng(8)
n, m, l, s = 130, 1000, 260, 520
G = I.random_k_body(rng, m, n, [1, 2, 3], 1); th = (0.3 * rng.normal(m, 2)).astype(np.float32)
A = I.bernoulli_bits(rng, l, n, 0.1, 3); Z = I.uniform_bits(rng, s, n, 4)
d = api.to_device_bits
ev, se = api.expval_raw(n, torch.from_numpy(th).cuda(), d(G), d(A), d(Z), "split_bf16")
wev, wse, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
al = rng.normal(l, 9) / s
g = api.expval_grad(n, torch.from_numpy(th).cuda(), d(G), d(A), d(Z), torch.from_numpy(al).cuda(), None, "split_bf16")
wg = oracle.expval_grad(n, G, A, Z, th.astype(np.float64), al, None)
print(json.dumps({"ev": float(np.max(np.abs(ev.cpu().numpy() - wev))), "se": float(np.max(np.abs(se.cpu().numpy() - wse))),
                  "g": float(np.linalg.norm(g.cpu().numpy() - wg) / np.linalg.norm(wg)), "status": api.read_status()}))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, IQP_CTA_PAIRS=pairs, IQP_SPLIT_TAIL=split, IQP_PHASE_TMEM=tmem, IQP_GRAD_PAIR=gpair,
               PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["status"] == 0
    assert r["ev"] <= TOL["split_bf16"] and r["se"] <= TOL["split_bf16"] and r["g"] <= GRAD_RTOL


def test_sixteen_warp_parity_gather_is_bit_exact():
    """The fused parity gather in CTAs of 16 warps (IQP_GATHER_WARPS=16: 512
    gates x 1024 rows per CTA) instead of 8: P and P^T bit-exact against the
    oracle on multi-tile ragged shapes, and the estimator that reads them,
    in a fresh process."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, numpy as np, torch, oracle
from paper_2501_04776_gb300 import api, inputs as I
d = api.to_device_bits
ok = True
for n, m, rows in [(200, 1100, 2100), (130, 1537, 1025), (777, 300, 129)]:
    rng = I.Rng(500 + n)
    R = I.bernoulli_bits(rng, rows, n, 0.5, 1)
    G = I.random_k_body(rng, m, n, [1, 2, 3], 2) if n != 777 else I.bernoulli_bits(rng, m, n, 0.5, 2)
    P, PT = api.parity_gather(n, d(R), d(G))
    want = oracle.parity(n, R, G)
    gP = I.unpack_bits(P.cpu().numpy().view(np.uint64), P.shape[1] * 64)
    gT = I.unpack_bits(PT.cpu().numpy().view(np.uint64), PT.shape[1] * 64)
    ok = ok and np.array_equal(gP[:, :m], want) and not gP[:, m:].any()
    ok = ok and np.array_equal(gT[:, :rows], want.T) and not gT[:, rows:].any()
rng = I.Rng(8)
n, m, l, s = 130, 1000, 260, 520
G = I.random_k_body(rng, m, n, [1, 2, 3], 1); th = (0.3 * rng.normal(m, 2)).astype(np.float32)
A = I.bernoulli_bits(rng, l, n, 0.1, 3); Z = I.uniform_bits(rng, s, n, 4)
ev, se = api.expval_raw(n, torch.from_numpy(th).cuda(), d(G), d(A), d(Z), "split_bf16")
wev, wse, _, _ = oracle.expval(n, G, A, Z, th.astype(np.float64))
print(json.dumps({"bits": bool(ok), "ev": float(np.max(np.abs(ev.cpu().numpy() - wev))),
                  "se": float(np.max(np.abs(se.cpu().numpy() - wse))), "status": api.read_status()}))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, IQP_GATHER_WARPS="16", PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["bits"] and r["status"] == 0
    assert r["ev"] <= TOL["split_bf16"] and r["se"] <= TOL["split_bf16"]

def test_two_sample_tile_phase_matches_single_tiles_and_oracle():
    """The split-BF16 phase of CTA pairs runs its full rounds as tiles of two
    256-sample tiles against each A stage (running sums in global memory) and
    the last round's double tiles as single tiles, split along the gates.
    On a shape with 88 double tiles for 76 CTA pairs and three accumulation
    chunks per tile, the fused statistics + gradient call agrees with the
    single-tile form (IQP_PHASE_DT=0) to FP32 rounding and, on sampled
    observables, with the oracle."""
    import os
    import subprocess
    import sys
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for dt in ("1", "0"):
        with tempfile.TemporaryDirectory() as tmp:
            path = os.path.join(tmp, "r.npz")
            env = dict(os.environ, IQP_PHASE_DT=dt, PYTHONPATH=root)
            r = subprocess.run([sys.executable, "-c", _TWO_TILE_CODE, path], env=env, cwd=root, capture_output=True,
                               text=True, timeout=600)
            assert r.returncode == 0, r.stderr[-2000:]
            z = np.load(path)
            out[dt] = {k: z[k] for k in ("ev", "se", "g", "status")}
    for dt in ("1", "0"):
        assert int(out[dt]["status"]) == 0
    # The two forms sum the gates in different orders (serpentine rounds
    # differ), so they agree to FP32 rounding of Phi and of the per-64-sample
    # cos statistics: 1e-6 of the estimates and of the standard errors. Each
    # gradient is about 2e-5 (relative) from the FP64 one, so two of them may
    # differ by that much; half the gradient tolerance bounds the difference.
    assert np.max(np.abs(out["1"]["ev"] - out["0"]["ev"])) <= 1e-6
    assert np.max(np.abs(out["1"]["se"] - out["0"]["se"])) <= 1e-7
    assert rel_l2(out["1"]["g"], out["0"]["g"]) <= GRAD_RTOL / 2
    n, G, A, Z, th, idx, al = _two_tile_problem()
    wev, wse, _, _ = oracle.expval(n, G, A[idx], Z, th.astype(np.float64))
    assert np.max(np.abs(out["1"]["ev"][idx] - wev)) <= TOL["split_bf16"]
    assert np.max(np.abs(out["1"]["se"][idx] - wse)) <= TOL["split_bf16"]
    wg = oracle.expval_grad(n, G, A[idx], Z, th.astype(np.float64), al[idx], None)
    assert rel_l2(out["1"]["g"], wg) <= GRAD_RTOL


def _two_tile_problem():
    """n=130, m=20000, l=2600 (11 observable blocks), s=3600 (8 double sample
    blocks); sampled observables on both sides of block edges."""
    rng = I.Rng(29)
    n, m, l, s = 130, 20000, 2600, 3600
    G = I.random_k_body(rng, m, n, [1, 2, 3], 1)
    th = (0.05 * rng.normal(m, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, 0.05, 3)
    Z = I.uniform_bits(rng, s, n, 4)
    idx = np.array([0, 1, 255, 256, 511, 1300, 2047, 2048, 2303, 2304, 2599])
    al = np.zeros(l)
    al[idx] = I.Rng(9).normal(idx.size, 1) / s
    return n, G, A, Z, th, idx, al


_TWO_TILE_CODE = """
import sys, numpy as np, torch
sys.path.insert(0, "tests")
from test_gpu import _two_tile_problem
from paper_2501_04776_gb300 import api
n, G, A, Z, th, idx, al = _two_tile_problem()
d = api.to_device_bits
ev, se, g = api.expval_value_and_grad(n, torch.from_numpy(th).cuda(), d(G), d(A), d(Z), torch.from_numpy(al).cuda(),
                                      None, "split_bf16")
np.savez(sys.argv[1], ev=ev.cpu().numpy(), se=se.cpu().numpy(), g=g.cpu().numpy(), status=api.read_status())
"""


# --------------------------------------------------------- bitflip circuits

@pytest.mark.parametrize("n,m,l", [(8, 36, 64), (130, 1000, 300), (131, 9000, 9000), (1000, 100_000, 257)])
def test_bitflip_expval_and_grad(api, n, m, l):
    """Stochastic bitflip circuit (Sec. 2.5): exact products and their
    gradient in FP64 against the oracle's product form / product rule."""
    import torch
    rng = I.Rng(60 + n)
    G = I.local_gates_packed(n) if n == 8 else I.random_k_body(rng, m, n, [1, 2, 3], 1)
    # angles small enough that the products over |J_a| ~ 0.1 m factors stay O(1)
    scale = {8: 0.15, 130: 0.1, 131: 0.03, 1000: 0.01}[n]
    th = (scale * rng.normal(G.shape[0], 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, 0.5 if n == 8 else 0.05, 3)
    if n >= 1000 or l > 1000:  # oracle on a subsample of observables: the gradient is linear in w
        idx = np.arange(0, l, 37 if n >= 1000 else 97)
    else:
        idx = np.arange(l)
    w = np.zeros(l)
    w[idx] = rng.normal(idx.size, 4)
    theta = th_dev(th).requires_grad_(True)
    ev = api.bitflip_expval(theta, dev(api, G), dev(api, A), n)
    (ev * torch.from_numpy(w).cuda()).sum().backward()
    want = oracle.bitflip_expval(n, G, A[idx], th.astype(np.float64))
    assert np.min(np.abs(want)) > 1e-3  # the check is not vacuous
    assert np.max(np.abs(ev.detach().cpu().numpy()[idx] - want)) <= 1e-12
    wg = oracle.bitflip_grad(n, G, A[idx], th.astype(np.float64), w[idx])
    g = theta.grad.double().cpu().numpy()
    # theta.grad is cast to theta's float32; compare the float64 result too.
    g64 = api.bitflip_grad(n, th_dev(th), dev(api, G), dev(api, A), torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel_l2(g64, wg) <= 1e-10
    assert rel_l2(g, wg) <= 1e-6


# ------------------------------------------------------- row-sparse form

def test_sparse_matches_dense_fp32_on_sparse_parities(api):
    """Low-density P_A (observables of weight ~4, one- and two-body gates):
    the row-sparse form agrees with the oracle and with the plain FP32 form,
    including observables whose P_A row is empty (<Z_a> = 1 exactly)."""
    p = I.mmd_training(seed=3, n=200, l=300, s=4100, N=10)
    p.theta = (p.theta * 20).astype(np.float32)
    p.A[:3] = 0  # a = 0: every phase is 0
    ev, se = gpu_expval(api, p, "sparse_fp32")
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev - want_ev)) <= TOL["sparse_fp32"]
    assert np.max(np.abs(se - want_se)) <= TOL["sparse_fp32"]
    assert np.all(ev[:3] == 1.0) and np.all(se[:3] == 0.0)
    ev32, _ = gpu_expval(api, p, "fp32")
    assert np.max(np.abs(ev - ev32)) <= 2 * TOL["fp32"]
    w = I.Rng(8).normal(p.l, 1)
    g = gpu_grad(api, p, -w / p.s, None, "sparse_fp32")
    want = oracle.expval_grad(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64), -w / p.s, None)
    assert rel_l2(g, want) <= GRAD_RTOL


def test_sparse_gradient_zero_weights_and_scale_extremes(api):
    """alpha = beta = 0 gives an exactly zero gradient; a tiny and a large
    weight scale give the same relative accuracy (the fixed-point scale is
    chosen per call)."""
    p = ragged_problem(seed=21, pa=0.02)
    assert np.array_equal(gpu_grad(api, p, np.zeros(p.l), None, "sparse_fp32"), np.zeros(p.m))
    w = I.Rng(9).normal(p.l, 1) / p.s
    want = oracle.expval_grad(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64), w, None)
    for f in (1e-30, 1.0, 1e30):
        g = gpu_grad(api, p, w * f, None, "sparse_fp32")
        assert rel_l2(g / f, want) <= GRAD_RTOL


# ------------------------------------------------------ value and gradient

@pytest.mark.parametrize("prec", PRECS)
def test_value_and_grad_matches_oracle(api, prec):
    """One call: estimates, standard errors and the gradient of a loss whose
    coefficients are known in advance (in split BF16 from a single pass of the
    phase contraction)."""
    import torch
    p = ragged_problem(seed=31)
    w = I.Rng(32).normal(p.l, 1)
    alpha = torch.from_numpy(-w / p.s).cuda()
    beta = torch.from_numpy(I.Rng(33).normal(p.l, 1) * 0.1 / p.s).cuda()
    ev, se, g = api.expval_value_and_grad(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z), alpha,
                                          beta, prec)
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev.cpu().numpy() - want_ev)) <= TOL[prec]
    assert np.max(np.abs(se.cpu().numpy() - want_se)) <= TOL[prec]
    want = oracle.expval_grad(p.n, p.G, p.A, p.Z, p.theta.astype(np.float64), -w / p.s,
                              beta.cpu().numpy())
    assert rel_l2(g.cpu().numpy(), want) <= GRAD_RTOL
    # the same numbers as the two separate calls (W is formed with the same
    # arithmetic from the same Phi, and every reduction has a fixed order)
    ev2, se2 = gpu_expval(api, p, prec)
    assert np.array_equal(ev.cpu().numpy(), ev2) and np.array_equal(se.cpu().numpy(), se2)
    assert np.array_equal(g.cpu().numpy(), gpu_grad(api, p, -w / p.s, beta.cpu().numpy(), prec))


def test_value_and_grad_full_size(api):
    """The benchmark workload (n=1000, m=1e5, l=s=1e4) in one call, sampled
    observables against the oracle on identical samples."""
    import torch
    p = I.random_gates(n=1000)
    idx = np.unique(np.sort(I.Rng(61).integers(8, p.l, 1)))
    alpha = np.zeros(p.l)
    alpha[idx] = I.Rng(62).normal(idx.size, 1) / p.s
    ev, se, g = api.expval_value_and_grad(p.n, th_dev(p.theta), dev(api, p.G), dev(api, p.A), dev(api, p.Z),
                                          torch.from_numpy(alpha).cuda(), None, "split_bf16")
    want_ev, want_se, _, _ = oracle.expval(p.n, p.G, p.A[idx], p.Z, p.theta.astype(np.float64))
    assert np.max(np.abs(ev.cpu().numpy()[idx] - want_ev)) <= TOL["split_bf16"]
    assert np.max(np.abs(se.cpu().numpy()[idx] - want_se)) <= TOL["split_bf16"]
    want = oracle.expval_grad(p.n, p.G, p.A[idx], p.Z, p.theta.astype(np.float64), alpha[idx], None)
    assert rel_l2(g.cpu().numpy(), want) <= GRAD_RTOL
