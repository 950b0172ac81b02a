"""Learned warm start: training pairs from the plain method, training, and the
warm-started solve.

Pairs: for seeded synthetic slices, input = the single-shot reconstruction
(ei_single_shot_fbp), target = the plain iterative reconstruction converged
to the relative-change tolerance, both in the solver's scaled units
u = x / scale (three channels, NHWC).  The network (ei.UNet) learns
target = input + net(input).  A warm-started solve runs the plain iteration
from the network's output to the same tolerance, so the warm start can save
iterations but never changes the stopping rule.

    python -m paper_2202_08627_gb300.warmstart --pairs 4096 --eval 256
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Sequence

import numpy as np

from . import ei, inputs, synth

SCALE = np.asarray(inputs.SCALE, dtype=np.float32)


def vol_to_u(G: ei.Geometry, vol):
    """vol layout (physical) of equal-size slices -> [S][n][n][3] in scaled units."""
    import torch
    n = G.slices[0].n
    sc = torch.as_tensor(SCALE, device=vol.device)
    return (vol.view(G.n_slices, n, n, 4)[..., :3] / sc).contiguous()


def u_to_vol(G: ei.Geometry, u, vol):
    import torch
    n = G.slices[0].n
    sc = torch.as_tensor(SCALE, device=u.device)
    v = vol.view(G.n_slices, n, n, 4)
    v[..., :3] = u * sc
    v[..., 3] = 0.0
    return vol


def net_forward_chunks(net: ei.UNet, x):
    import torch
    out = torch.empty_like(x)
    for b0 in range(0, x.shape[0], net.batch):
        out[b0:b0 + net.batch] = net.forward(x[b0:b0 + net.batch].contiguous())
    return out


def cnn_warm_start(net: ei.UNet, G: ei.Geometry, s_exp, vol_out):
    """vol_out = network(single-shot reconstruction), physical units."""
    ei.ei_single_shot_fbp(G, s_exp, vol_out)
    return u_to_vol(G, net_forward_chunks(net, vol_to_u(G, vol_out)), vol_out)


def generate_pairs(n_pairs: int, seed0: int, n: int = 256, n_theta: int = 720, n_det: int = 384,
                   n_m: int = 7, chunk: int = 64, tol: float = 1e-6, max_iter: int = 300,
                   device="cuda"):
    """(inputs, targets) [n_pairs][n][n][3] on the device, plus per-slice iteration counts."""
    import torch
    X = torch.empty((n_pairs, n, n, 3), dtype=torch.float32, device=device)
    Y = torch.empty_like(X)
    iters = []
    for c0 in range(0, n_pairs, chunk):
        k = min(chunk, n_pairs - c0)
        seeds = [seed0 + c0 + i for i in range(k)]
        G, s_exp = synth.build_problem([(n, n_theta, n_det)] * k, n_m, seeds, device, seed0 + c0)
        vol = G.empty("vol", device)
        ei.ei_single_shot_fbp(G, s_exp, vol)
        X[c0:c0 + k] = vol_to_u(G, vol)
        rep = ei.ei_reconstruct(G, s_exp, vol, tol=tol, max_iter=max_iter, raise_on_error=False)
        Y[c0:c0 + k] = vol_to_u(G, vol)
        iters += rep.iterations.tolist()
        G.close()
        del s_exp, vol
    return X, Y, np.asarray(iters)


def train(net: ei.UNet, X, Y, epochs: int, lr: float, seed: int = 0, lr_final: float | None = None):
    """Adam on mini-batches of net.batch shuffled pairs; returns the mean loss per epoch."""
    import torch
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    n = X.shape[0]
    hist = []
    steps = epochs * ((n + net.batch - 1) // net.batch)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(X.device)
        losses = []
        for b0 in range(0, n - net.batch + 1, net.batch):
            idx = perm[b0:b0 + net.batch]
            # cosine decay from lr to lr_final
            lr_t = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (
                1 + np.cos(np.pi * step / max(1, steps)))
            losses.append(net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr_t))
            step += 1
        hist.append(float(np.mean(losses)))
    return hist


def evaluate(net: ei.UNet, n_eval: int, seed0: int, n: int = 256, n_theta: int = 720,
             n_det: int = 384, n_m: int = 7, chunk: int = 64, tol: float = 1e-6,
             max_iter: int = 300, device="cuda"):
    """Time to tolerance of the held-out slices from x0 = 0, from the single-shot
    reconstruction and from the network's warm start (CUDA events around the
    start's computation and the solve)."""
    import torch
    res = {k: {"seconds": 0.0, "iterations": [], "f_final": []}
           for k in ("zero", "single_shot", "cnn")}
    for c0 in range(0, n_eval, chunk):
        k = min(chunk, n_eval - c0)
        seeds = [seed0 + c0 + i for i in range(k)]
        G, s_exp = synth.build_problem([(n, n_theta, n_det)] * k, n_m, seeds, device, seed0 + c0)
        for start in res:
            vol = G.empty("vol", device)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if start == "single_shot":
                ei.ei_single_shot_fbp(G, s_exp, vol)
            elif start == "cnn":
                cnn_warm_start(net, G, s_exp, vol)
            rep = ei.ei_reconstruct(G, s_exp, vol, tol=tol, max_iter=max_iter, raise_on_error=False)
            e1.record()
            torch.cuda.synchronize()
            res[start]["seconds"] += e0.elapsed_time(e1) * 1e-3
            res[start]["iterations"] += rep.iterations.tolist()
            res[start]["f_final"] += rep.f_final.tolist()
        G.close()
    eq = n_eval * (n / 1024.0) ** 2
    out = {}
    for k, v in res.items():
        it = np.asarray(v["iterations"])
        out[k] = {"seconds": v["seconds"], "seconds_per_1024_slice": v["seconds"] / eq,
                  "iterations_mean": float(it.mean()), "iterations_median": float(np.median(it)),
                  "iterations_max": int(it.max()), "f_final_mean": float(np.mean(v["f_final"]))}
    zf = np.asarray(res["zero"]["f_final"])
    cf = np.asarray(res["cnn"]["f_final"])
    out["cnn_vs_zero_f_final_rel_diff_max"] = float(np.max(np.abs(cf - zf) / np.abs(zf)))
    return out


def main(argv: Sequence[str] | None = None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--eval", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    X, Y, it = generate_pairs(args.pairs, 1_000_000, n=args.size)
    t1 = time.time()
    net = ei.UNet(levels=args.levels, base=args.base, batch=args.batch, height=args.size,
                  width=args.size, seed=0)
    hist = train(net, X, Y, args.epochs, args.lr, lr_final=args.lr * 0.05)
    torch.cuda.synchronize()
    t2 = time.time()
    if args.save:
        np.save(args.save, net.get_params())
    ev = evaluate(net, args.eval, 2_000_000, n=args.size)
    print(json.dumps({"pairs": args.pairs, "pair_generation_s": t1 - t0, "training_s": t2 - t1,
                      "pair_iterations_mean": float(it.mean()), "loss_per_epoch": hist,
                      "eval": ev}))


if __name__ == "__main__":
    main()
