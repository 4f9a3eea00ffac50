"""iqp_expval_noalloc: the forward estimator for callers that cannot allocate
device memory at call time (their device memory is owned by another
framework's pool, or cudaMalloc's synchronisation is too slow for them). It
keeps its scratch in a fixed 64 MiB device array inside the library instead
of a caller workspace. Checked through the C ABI against iqp_expval on the
same inputs, in every precision, on two calls in a row (different shapes, so
stale contents of the shared array would show), for its device status word
(iqp_noalloc_read_status), its argument checks and its size limit.

Both entry points run the same kernels on the same inputs, so the results
must agree bit for bit, not only within the parity tolerances.

This file is collected last on purpose; it also passes alone in a fresh
process (it builds and loads the library itself)."""
import ctypes

import numpy as np
import pytest

from paper_2501_04776_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem(seed, n, m, l, s, ks=(1, 2, 3)):
    rng = I.Rng(seed)
    G = I.random_k_body(rng, m, n, list(ks), 1)
    theta = (0.3 * rng.normal(m, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, 0.1, 3)
    Z = I.uniform_bits(rng, s, n, 4)
    return n, G, A, Z, theta


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2501_04776_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    assert torch.cuda.is_available()
    return torch, _lib, lib


def _run(env, prob, prec, noalloc):
    torch, _lib, lib = env
    n, G, A, Z, theta = prob
    dev = lambda w: torch.from_numpy(np.ascontiguousarray(w).view(np.int64)).cuda()
    Gd, Ad, Zd = dev(G), dev(A), dev(Z)
    th = torch.from_numpy(theta).cuda()
    m, l, s = G.shape[0], A.shape[0], Z.shape[0]
    ev = torch.full((l,), float("nan"), dtype=torch.float64, device="cuda")
    se = torch.full((l,), float("nan"), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    args = (n, P(Gd), m, Gd.shape[1], P(Ad), l, Ad.shape[1], P(Zd), s, Zd.shape[1], P(th), prec, P(ev), P(se))
    if noalloc:
        rc = lib.iqp_expval_noalloc(*args, st)
        assert rc == _lib.OK, _lib.status_string(rc)
        status = lib.iqp_noalloc_read_status(st)
    else:
        nbytes = lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, prec)
        ws = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")  # status word starts at zero
        rc = lib.iqp_expval(*args, P(ws), nbytes, st)
        assert rc == _lib.OK, _lib.status_string(rc)
        status = lib.iqp_read_status(P(ws), nbytes, st)
    assert status == _lib.OK, _lib.status_string(status)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), se.cpu().numpy()


# FP32, split BF16, row-sparse FP32 (integer accumulators), low-order FP32
# (generators of weight <= 2; fixed-point sums in its scratch).
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_workspace_entry_point_twice(env, prec):
    ks = (1, 2) if prec == 3 else (1, 2, 3)
    first = _problem(31, 130, 1000, 300, 600, ks)
    second = _problem(32, 70, 333, 129, 257, ks)
    for prob in (first, second):
        want_ev, want_se = _run(env, prob, prec, noalloc=False)
        got_ev, got_se = _run(env, prob, prec, noalloc=True)
        assert np.all(np.isfinite(got_ev)) and np.all(np.isfinite(got_se))
        assert np.array_equal(got_ev, want_ev)
        assert np.array_equal(got_se, want_se)


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, _lib, lib = env
    n, m, l, s = 1000, 100_000, 10_000, 10_000  # needs ~250 MB of scratch
    assert lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, 1) > (64 << 20)
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.iqp_expval_noalloc(n, p, m, 16, p, l, 16, p, s, 16, p, 1, p, p,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.ERR_WORKSPACE


def test_noalloc_argument_errors_match_iqp_expval(env):
    """Invalid arguments give iqp_expval's status (checked before the size
    limit and before anything is queued)."""
    torch, _lib, lib = env
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = ctypes.c_void_p(buf.data_ptr())
    for n, m, prec in ((0, 10, 1), (64, 0, 1), (64, 10, 7)):
        want = lib.iqp_expval(n, p, m, 2, p, 4, 2, p, 4, 2, p, prec, p, p, ws, buf.numel(), st)
        got = lib.iqp_expval_noalloc(n, p, m, 2, p, 4, 2, p, 4, 2, p, prec, p, p, st)
        assert got == want == _lib.ERR_ARG
    assert lib.iqp_noalloc_read_status(st) == _lib.OK
