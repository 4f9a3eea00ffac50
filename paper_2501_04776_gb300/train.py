"""Plain Adam loop on the MMD^2 loss (Sec. 3.3.1 with the training procedure of
Sec. 2.4: a fresh sample batch Z, and fresh observables a ~ P_sigma, at every
step; the data set is fixed). Loss and gradient come from one call of
iqp_mmd_loss_grad per step; the Adam update is ordinary PyTorch.

    python -m paper_2501_04776_gb300.train --n 1000 --steps 50

trains the one- and two-body circuit on n qubits (m = n(n+1)/2 gates) against
10000 rows drawn from 8 prototype bitstrings with 5% flips, with 2000
observables and 5000 samples per step, and prints one JSON line per step.
With --cuda-graph each step after the third replays its loss, backward and
Adam update from one CUDA graph (observables and samples drawn on the device).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import api, inputs as I


def choose_precision(G: np.ndarray) -> str:
    """The low-order form when every generator acts on at most two qubits
    (checked on the host from the packed rows), else split BF16."""
    wt = np.bitwise_count(np.ascontiguousarray(G, dtype=np.uint64)).sum(axis=1)
    return "loworder_fp32" if wt.size and int(wt.max()) <= 2 else "split_bf16"


def adam_mmd(problem: I.Problem, steps: int, lr: float = 1e-3, precision: str = "auto",
             unbiased: bool = True, seed: int = 0, device: str = "cuda", log=None, device_rng: bool = False,
             sqrt_loss: bool = False, indep: bool = False, cuda_graph: bool = False):
    """Returns (theta, losses). problem.A / problem.Z give the observable and
    sample counts; fresh ones are drawn every step from seed: on the host
    (inputs.fresh_*) or, with device_rng, by the library's on-device generator
    (bit-identical draws). indep draws l * s samples per step, one batch per
    observable; sqrt_loss trains on sqrt(MMD^2).

    cuda_graph (needs device_rng): the first steps run eagerly, then the loss,
    its backward and the Adam update of one step are captured in a CUDA graph
    that every later step replays after drawing its observables and samples
    into the captured buffers (the step's ~30 short launches become one)."""
    if cuda_graph:
        return _adam_mmd_graph(problem, steps, lr, precision, unbiased, seed, device, log, sqrt_loss, indep)
    n = problem.n
    l, s = problem.A.shape[0], problem.Z.shape[0]
    if precision == "auto":
        precision = choose_precision(problem.G)
    ps = problem.extra.get("p_sigma", 0.5)
    G = api.to_device_bits(problem.G, device)
    X = api.to_device_bits(problem.X, device)
    theta = torch.nn.Parameter(torch.from_numpy(problem.theta.astype(np.float32)).to(device))
    opt = torch.optim.Adam([theta], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    for step in range(steps):
        t0 = time.perf_counter()
        zrows = l * s if indep else s
        if device_rng:
            A = api.bernoulli_bits(seed, 1001 + 2 * step, l, n, ps, device)
            Z = api.uniform_bits(seed, 1000 + 2 * step, zrows, n, device)
        else:
            A = api.to_device_bits(I.fresh_observables(seed, step, l, n, ps), device)
            Z = api.to_device_bits(I.fresh_samples(seed, step, zrows, n), device)
        opt.zero_grad(set_to_none=True)
        loss = api.mmd_loss(theta, G, A, Z, X, n, precision, unbiased, sqrt_loss, indep)
        loss.backward()
        opt.step()
        lv = float(loss.detach())
        losses.append(lv)
        if log is not None:
            torch.cuda.synchronize()
            log({"step": step, "loss": lv, "ms": round(1e3 * (time.perf_counter() - t0), 3)})
    return theta.detach(), losses


def _adam_mmd_graph(problem, steps, lr, precision, unbiased, seed, device, log, sqrt_loss, indep, warm=3):
    n = problem.n
    l, s = problem.A.shape[0], problem.Z.shape[0]
    if precision == "auto":
        precision = choose_precision(problem.G)
    ps = problem.extra.get("p_sigma", 0.5)
    G = api.to_device_bits(problem.G, device)
    X = api.to_device_bits(problem.X, device)
    zrows = l * s if indep else s
    ld = api.words_per_row(n)
    A = torch.empty(l, ld, dtype=torch.int64, device=device)
    Z = torch.empty(zrows, ld, dtype=torch.int64, device=device)
    theta = torch.nn.Parameter(torch.from_numpy(problem.theta.astype(np.float32)).to(device))
    opt = torch.optim.Adam([theta], lr=lr, betas=(0.9, 0.999), eps=1e-8, capturable=True)

    def draw(step):
        api.bernoulli_bits(seed, 1001 + 2 * step, l, n, ps, device, out=A)
        api.uniform_bits(seed, 1000 + 2 * step, zrows, n, device, out=Z)

    def train_step():
        opt.zero_grad(set_to_none=False)
        loss = api.mmd_loss(theta, G, A, Z, X, n, precision, unbiased, sqrt_loss, indep)
        loss.backward()
        opt.step()
        return loss

    losses, graph, static_loss = [], None, None
    side = torch.cuda.Stream(device)
    for step in range(steps):
        t0 = time.perf_counter()
        if step < warm:
            side.wait_stream(torch.cuda.current_stream(device))
            with torch.cuda.stream(side):  # eager steps on a side stream, as capture wants
                draw(step)
                loss = train_step()
            torch.cuda.current_stream(device).wait_stream(side)
        else:
            if graph is None:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    static_loss = train_step()
            draw(step)
            graph.replay()
            loss = static_loss
        lv = float(loss.detach())
        losses.append(lv)
        if log is not None:
            torch.cuda.synchronize()
            log({"step": step, "loss": lv, "ms": round(1e3 * (time.perf_counter() - t0), 3)})
    return theta.detach(), losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--l", type=int, default=2000)
    ap.add_argument("--s", type=int, default=5000)
    ap.add_argument("--N", type=int, default=10_000)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--precision", default="auto", choices=["auto", "split_bf16", "fp32", "sparse_fp32", "loworder_fp32"])
    ap.add_argument("--device-rng", action="store_true", help="draw samples and observables on the GPU")
    ap.add_argument("--sqrt-loss", action="store_true")
    ap.add_argument("--indep", action="store_true", help="one sample batch per observable")
    ap.add_argument("--cuda-graph", action="store_true",
                    help="replay each step's loss, backward and Adam update from a CUDA graph (needs --device-rng)")
    args = ap.parse_args()
    p = I.mmd_training(n=args.n, l=args.l, s=args.s, N=args.N)
    print(json.dumps({"workload": p.name, "p_sigma": p.extra["p_sigma"], "m": p.m}), flush=True)
    _, losses = adam_mmd(p, args.steps, args.lr, args.precision, log=lambda r: print(json.dumps(r), flush=True),
                         device_rng=args.device_rng or args.cuda_graph, sqrt_loss=args.sqrt_loss, indep=args.indep,
                         cuda_graph=args.cuda_graph)
    print(json.dumps({"first_loss": losses[0], "last_loss": losses[-1],
                      "mean_first5": float(np.mean(losses[:5])), "mean_last5": float(np.mean(losses[-5:]))}))


if __name__ == "__main__":
    main()
