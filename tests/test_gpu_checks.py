"""The self-checked build (-DIQP_CHECKS): every kernel compares each global
index it derives from the caller's shapes with its buffer's extent, records a
failure in a check word and skips the access (it never traps). This test
builds that variant beside the default library and, in a fresh process that
loads it, runs every entry point on ragged small problems: the check words
and the workspace status must stay 0, and the results must still match the
FP64 oracle at the parity tolerances (so the checks reject nothing valid)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, numpy as np, torch, oracle
from paper_2501_04776_gb300 import api, _lib, inputs as I
lib = _lib.load()
assert lib.iqp_checks_enabled() == 1
out = {"errors": {}, "status": {}}
TOL = {"fp32": 1e-5, "split_bf16": 1e-4, "sparse_fp32": 1e-5, "loworder_fp32": 1e-5}
d = api.to_device_bits
th = lambda t: torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()
rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

def record(tag):
    torch.cuda.synchronize()
    out["status"][tag] = [int(api.read_status()), int(lib.iqp_check_status())]

def problem(seed, n, m, l, s, ks):
    rng = I.Rng(seed)
    G = I.random_k_body(rng, m, n, list(ks), 1)
    theta = (0.3 * rng.normal(m, 2)).astype(np.float32)
    A = I.bernoulli_bits(rng, l, n, 0.1, 3)
    Z = I.uniform_bits(rng, s, n, 4)
    return n, G, A, Z, theta

for prec in ("fp32", "split_bf16", "sparse_fp32", "loworder_fp32"):
    for shape in ((130, 1000, 300, 600), (70, 333, 129, 257)):
        n, G, A, Z, theta = problem(11, *shape, (1, 2) if prec == "loworder_fp32" else (1, 2, 3))
        l, s = A.shape[0], Z.shape[0]
        ev, se = api.expval_raw(n, th(theta), d(G), d(A), d(Z), prec)
        wev, wse, _, _ = oracle.expval(n, G, A, Z, theta.astype(np.float64))
        al = I.Rng(5).normal(l, 1) / s
        g = api.expval_grad(n, th(theta), d(G), d(A), d(Z), torch.from_numpy(al).cuda(), None, prec)
        wg = oracle.expval_grad(n, G, A, Z, theta.astype(np.float64), al, None)
        ev2, se2, g2 = api.expval_value_and_grad(n, th(theta), d(G), d(A), d(Z), torch.from_numpy(al).cuda(), None, prec)
        tag = f"{prec}-{shape}"
        out["errors"][tag] = {"ev": float(np.max(np.abs(ev.cpu().numpy() - wev))),
                              "se": float(np.max(np.abs(se.cpu().numpy() - wse))),
                              "g": rel(g.cpu().numpy(), wg), "g2": rel(g2.cpu().numpy(), wg),
                              "tol": TOL[prec]}
        record(tag)
        if prec != "fp32":
            phi = api.expval_keep_phi_raw(n, th(theta), d(G), d(A), d(Z), prec)[2]
            g3 = api.expval_grad_from_phi(n, th(theta), d(G), d(A), d(Z), phi, torch.from_numpy(al).cuda(), None, prec)
            out["errors"][tag]["g3"] = rel(g3.cpu().numpy(), wg)
            record(tag + "-kept")

# A shape whose split-BF16 phase runs full rounds of two-sample tiles and the
# last round as single tiles and split parts (88 double tiles for 76 pairs):
# sampled observables against the oracle
n, G, A, Z, theta = problem(17, 130, 20000, 2600, 3600, (1, 2, 3))
theta = (theta / 6).astype(np.float32)
idx = np.array([0, 255, 256, 1300, 2303, 2304, 2599])
ev, se = api.expval_raw(n, th(theta), d(G), d(A), d(Z), "split_bf16")
wev, wse, _, _ = oracle.expval(n, G, A[idx], Z, theta.astype(np.float64))
out["errors"]["two-tile"] = {"ev": float(np.max(np.abs(ev.cpu().numpy()[idx] - wev))),
                             "se": float(np.max(np.abs(se.cpu().numpy()[idx] - wse))), "tol": TOL["split_bf16"]}
record("two-tile")

# MMD loss and gradient (shared and independent batches), bitflip, parities, variants
rng = I.Rng(3)
n, G, A, Z, theta = problem(21, 60, 400, 120, 300, (1, 2, 3))
X = I.prototype_data(rng, 200, n, 4, 0.05, 9)
for prec in ("split_bf16", "sparse_fp32"):
    loss, grad = api.mmd_loss_raw(n, th(theta), d(G), d(A), d(Z), d(X), prec, True, with_grad=True)
    wl, _, wg = oracle.mmd_loss(n, G, A, Z, X, theta.astype(np.float64), True, grad=True)
    out["errors"]["mmd-" + prec] = {"loss": abs(float(loss) - wl), "g": rel(grad.cpu().numpy(), wg), "tol": TOL[prec]}
    record("mmd-" + prec)
Zi = I.uniform_bits(rng, A.shape[0] * 64, n, 12)
evi, sei = api.expval_indep_raw(n, th(theta), d(G), d(A), d(Zi))
record("indep")
evb = api.bitflip_expval_raw(n, th(theta), d(G), d(A))
gb = api.bitflip_grad(n, th(theta), d(G), d(A), torch.ones(A.shape[0], dtype=torch.float64, device="cuda"))
record("bitflip")
P = api.parity(n, d(Z), d(G))
PT = api.parity_gather(n, d(Z), d(G))
T = api.parity_sum(n, d(A), d(X))
want = oracle.parity(n, Z, G)
Pw = P.cpu().numpy().view(np.uint64)
got = I.unpack_bits(Pw, Pw.shape[1] * 64)
out["errors"]["parity"] = {"mismatch": int(np.count_nonzero(got[:, :G.shape[0]] != want)), "tol": 0}
record("parity")
api.uniform_bits(1, 2, 77, n)
api.bernoulli_bits(1, 3, 77, n, 0.2)
api.embed_bits(d(A), n, list(range(0, 2 * n, 2))[:n], 2 * n)
start = np.array([0, 3, 3, 10, G.shape[0]], dtype=np.int64)
api.expand_params(th(np.arange(4, dtype=np.float32)), start, G.shape[0])
record("variants")
print(json.dumps(out))
'''


def test_self_checked_build_records_nothing_and_matches_oracle():
    from paper_2501_04776_gb300 import build
    build.build(checks=True)
    env = dict(os.environ, IQP_CHECKED_LIB="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for tag, (status, check) in out["status"].items():
        assert status == 0 and check == 0, (tag, status, check)
    for tag, e in out["errors"].items():
        tol = e["tol"]
        if tag == "parity":
            assert e["mismatch"] == 0
            continue
        for k, v in e.items():
            if k == "tol":
                continue
            bound = 1e-4 if k.startswith("g") else tol  # gradients: relative L2
            assert v <= bound, (tag, k, v)
