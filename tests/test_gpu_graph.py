"""The library's calls inside a CUDA graph: an expval-and-gradient call and an
MMD^2 loss-and-gradient call are captured once (after warm-up calls on the
capture stream) and replayed; the replays give the eager results bit for bit,
and the graph follows new inputs copied into the captured buffers. The Adam
training loop replays its captured step on fresh draws like the eager loop."""
import numpy as np
import pytest

import oracle
from paper_2501_04776_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2501_04776_gb300 import build
    build.build()
    from paper_2501_04776_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def capture(fn, warmup=2):
    """Warm fn up on a side stream, capture one call into a graph; returns
    (graph, outputs of the captured call)."""
    import torch
    from paper_2501_04776_gb300 import _lib
    _lib.load().iqp_profile_enable(0)  # per-launch timing events have no place in a graph
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = fn()
    return g, out


@pytest.mark.parametrize("prec", ["split_bf16", "loworder_fp32"])
def test_value_and_grad_replays_bit_for_bit(api, prec):
    import torch
    rng = I.Rng(41)
    n, l, s = 48, 96, 700
    G = I.local_gates_packed(n)
    m = G.shape[0]
    th = (0.3 * rng.normal(m, 1) / np.sqrt(n)).astype(np.float32)
    A, Z = I.bernoulli_bits(rng, l, n, 0.15, 2), I.uniform_bits(rng, s, n, 3)
    Gd, Ad, Zd = (api.to_device_bits(x) for x in (G, A, Z))
    thd = torch.from_numpy(th).cuda()
    alpha = torch.from_numpy(rng.normal(l, 4) / s).cuda()

    def call():
        return api.expval_value_and_grad(n, thd, Gd, Ad, Zd, alpha, None, prec)

    eager = [t.clone() for t in call()]
    g, out = capture(call)
    for t in out:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, eager):
        assert torch.equal(a, b)
    # new samples and angles through the same graph
    Z2 = I.uniform_bits(rng, s, n, 5)
    th2 = (0.3 * rng.normal(m, 6) / np.sqrt(n)).astype(np.float32)
    Zd.copy_(api.to_device_bits(Z2))
    thd.copy_(torch.from_numpy(th2).cuda())
    g.replay()
    torch.cuda.synchronize()
    want_ev, _, _, _ = oracle.expval(n, G, A, Z2, th2.astype(np.float64))
    tol = 1e-4 if prec == "split_bf16" else 1e-5
    assert np.max(np.abs(out[0].cpu().numpy() - want_ev)) <= tol
    want_g = oracle.expval_grad(n, G, A, Z2, th2.astype(np.float64), alpha.cpu().numpy())
    got_g = out[2].cpu().numpy()
    assert np.linalg.norm(got_g - want_g) <= 1e-4 * np.linalg.norm(want_g)


def test_mmd_loss_grad_replays_bit_for_bit(api):
    import torch
    p = I.mmd_training(seed=21, n=60, l=150, s=600, N=400)
    Gd, Ad, Zd, Xd = (api.to_device_bits(x) for x in (p.G, p.A, p.Z, p.X))
    thd = torch.from_numpy((p.theta * 20).astype(np.float32)).cuda()

    def call():
        return api.mmd_loss_raw(p.n, thd, Gd, Ad, Zd, Xd, "loworder_fp32", True, with_grad=True)

    loss0, grad0 = (t.clone() for t in call())
    g, (loss, grad) = capture(call)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(loss, loss0) and torch.equal(grad, grad0)
    wl, _, wg = oracle.mmd_loss_ex(p.n, p.G, p.A, p.Z, p.X, (p.theta * 20).astype(np.float32).astype(np.float64),
                                   True, False, grad=True)
    assert abs(float(loss) - wl) <= 1e-5
    assert np.linalg.norm(grad.cpu().numpy() - wg) <= 1e-4 * np.linalg.norm(wg)


def test_training_loop_in_a_cuda_graph_follows_the_eager_loop(api):
    """adam_mmd with cuda_graph: three eager steps, then every step replays
    the captured loss, backward and Adam update on freshly drawn observables
    and samples. The same loop run eagerly throughout (the same capturable
    Adam) gives the same losses bit for bit; the default eager loop (Adam's
    non-capturable form, which rounds its update differently) stays within a
    relative 1e-4 over these steps."""
    from paper_2501_04776_gb300 import train
    p = I.mmd_training(seed=22, n=40, l=120, s=400, N=300)
    args = (p, 8, 1e-2, "loworder_fp32", True, 0, "cuda", None, False, False)
    _, graph = train._adam_mmd_graph(*args, warm=3)
    _, eager_same = train._adam_mmd_graph(*args, warm=8)
    assert graph == eager_same
    _, eager = train.adam_mmd(p, 8, lr=1e-2, precision="loworder_fp32", device_rng=True)
    assert np.allclose(graph, eager, rtol=1e-4, atol=1e-9)
    assert graph[-1] < graph[0]
