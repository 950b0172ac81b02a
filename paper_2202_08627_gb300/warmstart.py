"""Learned warm start: training pairs from the plain method, training, and the
warm-started solve.

Pairs: for seeded synthetic slices, input = the single-shot reconstruction
(ei_single_shot_fbp), target = the plain iterative reconstruction converged
to the relative-change tolerance, both in the solver's scaled units
u = x / scale (three channels, NHWC).  The network (ei.UNet) learns
target = input + net(input).  It is fully convolutional: it trains on square
crops of the pairs (offsets on the pooling grid) and runs on whole slices of
any size its pooling divides, one network instance per slice size sharing
the trained parameters.  A warm-started solve runs the plain iteration from
the network's output to the same tolerance, so the warm start can save
iterations but never changes the stopping rule.

    python -m paper_2202_08627_gb300.warmstart --pairs 4096 --eval 256
    python -m paper_2202_08627_gb300.warmstart --shapes uneven1024 --pairs 256 --eval 256
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import ei, inputs, synth

SCALE = np.asarray(inputs.SCALE, dtype=np.float32)


# ------------------------------------------------------------------ layout
def size_groups(G: ei.Geometry) -> Dict[int, List[int]]:
    """Slice indices grouped by slice size n."""
    groups: Dict[int, List[int]] = {}
    for s, sl in enumerate(G.slices):
        groups.setdefault(sl.n, []).append(s)
    return groups


def _slice_view(G: ei.Geometry, vol, s: int):
    sl = G.slices[s]
    return vol[sl.vol_offset:sl.vol_offset + sl.vol_count].view(sl.n, sl.n, 4)


def vol_to_u(G: ei.Geometry, vol, idx: Sequence[int] | None = None):
    """Slices idx (equal size; default all) of a vol-layout tensor -> [k][n][n][3]
    in scaled units."""
    import torch
    idx = range(G.n_slices) if idx is None else idx
    sc = torch.as_tensor(SCALE, device=vol.device)
    return torch.stack([_slice_view(G, vol, s)[..., :3] / sc for s in idx]).contiguous()


def u_to_vol(G: ei.Geometry, u, vol, idx: Sequence[int] | None = None):
    """Inverse of vol_to_u: writes physical units (fourth component 0) into vol."""
    import torch
    idx = range(G.n_slices) if idx is None else idx
    sc = torch.as_tensor(SCALE, device=u.device)
    for k, s in enumerate(idx):
        v = _slice_view(G, vol, s)
        v[..., :3] = u[k] * sc
        v[..., 3] = 0.0
    return vol


# ------------------------------------------------------------------ network
class WarmStartNet:
    """Trained parameters plus one inference instance of the network per slice
    size (created on first use, parameters copied in)."""

    def __init__(self, levels: int = 4, base: int = 32, crop: int = 256, batch: int = 16,
                 seed: int = 0):
        self.levels, self.base, self.crop, self.batch = levels, base, crop, batch
        self.train_net = ei.UNet(levels=levels, base=base, batch=batch, height=crop, width=crop,
                                 seed=seed)
        self._infer: Dict[int, ei.UNet] = {}
        self._version = 0
        self._loaded: Dict[int, int] = {}

    @property
    def granule(self) -> int:
        return 1 << (self.levels - 1)

    def mark_trained(self):
        self._version += 1

    def net_for(self, n: int) -> ei.UNet:
        if n % self.granule:
            raise ValueError("slice size %d is not a multiple of %d" % (n, self.granule))
        if n == self.crop:
            return self.train_net
        if n not in self._infer:
            # four times the training batch's pixels per forward (measured per
            # 1024^2 image: 4.08 ms at batch 1, 3.56 ms at batch 4; per 512^2
            # image: 1.02 ms at 4, 0.89 ms at 16); every image's output is the
            # same at any batch
            b = max(1, min(16, (4 * self.crop * self.crop * self.batch) // (n * n)))
            self._infer[n] = ei.UNet(levels=self.levels, base=self.base, batch=b, height=n,
                                     width=n, seed=0)
        if self._loaded.get(n) != self._version:
            self._infer[n].set_params(self.train_net.get_params())
            self._loaded[n] = self._version
        return self._infer[n]

    def apply(self, u):
        """u [k][n][n][3] -> network output, in chunks of the instance's batch."""
        import torch
        net = self.net_for(u.shape[1])
        out = torch.empty_like(u)
        for b0 in range(0, u.shape[0], net.batch):
            out[b0:b0 + net.batch] = net.forward(u[b0:b0 + net.batch].contiguous())
        return out

    def save(self, path: str):
        np.save(path, self.train_net.get_params())

    def load(self, path: str):
        self.train_net.set_params(np.load(path))
        self.mark_trained()

    def close(self):
        for net in self._infer.values():
            net.close()
        self._infer.clear()
        self.train_net.close()


def cnn_warm_start(net: WarmStartNet, G: ei.Geometry, s_exp, vol_out):
    """vol_out = network(single-shot reconstruction) for every slice, physical units."""
    ei.ei_single_shot_fbp(G, s_exp, vol_out)
    for n, idx in size_groups(G).items():
        u_to_vol(G, net.apply(vol_to_u(G, vol_out, idx)), vol_out, idx)
    return vol_out


# ------------------------------------------------------------------ pairs
def generate_pairs(shapes: Sequence[Tuple[int, int, int]], seed0: int, n_m: int = 7,
                   max_chunk_voxels: int = 64 * 256 * 256, tol: float = 1e-6,
                   max_iter: int = 400, device="cuda"):
    """Training pairs for slices of the given (n, n_theta, n_det), seeds seed0 + i.
    Returns ({n: (X, Y)} with X, Y [k][n][n][3] on the device, iteration counts)."""
    import torch
    xs: Dict[int, list] = {}
    ys: Dict[int, list] = {}
    iters = []
    i = 0
    while i < len(shapes):
        j, vox = i, 0
        while j < len(shapes) and (j == i or vox + shapes[j][0] ** 2 <= max_chunk_voxels):
            vox += shapes[j][0] ** 2
            j += 1
        chunk = list(shapes[i:j])
        seeds = [seed0 + k for k in range(i, j)]
        G, s_exp = synth.build_problem(chunk, n_m, seeds, device, seed0 + i)
        vol = G.empty("vol", device)
        ei.ei_single_shot_fbp(G, s_exp, vol)
        groups = size_groups(G)
        X = {n: vol_to_u(G, vol, idx) for n, idx in groups.items()}
        rep = ei.ei_reconstruct(G, s_exp, vol, tol=tol, max_iter=max_iter, raise_on_error=False)
        for n, idx in groups.items():
            xs.setdefault(n, []).append(X[n])
            ys.setdefault(n, []).append(vol_to_u(G, vol, idx))
        iters += rep.iterations.tolist()
        G.close()
        del s_exp, vol
        i = j
    pairs = {n: (torch.cat(xs[n]), torch.cat(ys[n])) for n in xs}
    return pairs, np.asarray(iters)


# ------------------------------------------------------------------ training
def train(net: WarmStartNet, pairs: Dict[int, tuple], epochs: int, lr: float, seed: int = 0,
          lr_final: float | None = None, steps_per_epoch: int | None = None):
    """Adam on mini-batches of crops (net.crop square, offsets multiples of the
    pooling granule) drawn uniformly over all crop positions of all pairs;
    cosine decay from lr to lr_final.  Returns the mean loss per epoch."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    c, g, B = net.crop, net.granule, net.batch
    sizes = sorted(pairs)
    for n in sizes:
        if n < c:
            raise ValueError("pairs of size %d are smaller than the crop %d" % (n, c))
    # weight each size by its number of crop positions
    npos = {n: ((n - c) // g + 1) ** 2 for n in sizes}
    w = np.array([pairs[n][0].shape[0] * npos[n] for n in sizes], dtype=np.float64)
    w /= w.sum()
    total_crops = sum(pairs[n][0].shape[0] * (n // c) ** 2 for n in sizes)
    spe = steps_per_epoch or max(1, total_crops // B)
    steps = epochs * spe
    dev = pairs[sizes[0]][0].device
    xb = torch.empty((B, c, c, 3), dtype=torch.float32, device=dev)
    yb = torch.empty_like(xb)
    hist, step = [], 0
    for ep in range(epochs):
        losses = []
        for _ in range(spe):
            for b in range(B):
                n = sizes[int(rng.choice(len(sizes), p=w))]
                X, Y = pairs[n]
                k = int(rng.integers(X.shape[0]))
                y0 = int(rng.integers((n - c) // g + 1)) * g
                x0 = int(rng.integers((n - c) // g + 1)) * g
                xb[b] = X[k, y0:y0 + c, x0:x0 + c]
                yb[b] = Y[k, y0:y0 + c, x0:x0 + c]
            lr_t = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (
                1 + np.cos(np.pi * step / max(1, steps)))
            losses.append(net.train_net.train_step(xb, yb, lr_t))
            step += 1
        hist.append(float(np.mean(losses)))
    net.mark_trained()
    return hist


# ------------------------------------------------------------------ evaluation
def time_to_tolerance(G: ei.Geometry, s_exp, starts: Sequence[str], tol: float, max_iter: int,
                      net: WarmStartNet | None = None):
    """Solve every slice to the relative-change tolerance from each start
    ("zero", "single_shot", "cnn"); CUDA events around the start's computation
    and the solve.  Per start: seconds, seconds per 1024^2-voxel slice,
    iteration statistics, converged count and final objectives."""
    import torch
    eq = sum(sl.n * sl.n for sl in G.slices) / 1024.0 ** 2
    out = {}
    for start in starts:
        vol = G.empty("vol", s_exp.device)
        torch.cuda.synchronize()
        e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        if start == "single_shot":
            ei.ei_single_shot_fbp(G, s_exp, vol)
        elif start == "cnn":
            cnn_warm_start(net, G, s_exp, vol)
        elif start != "zero":
            raise ValueError(start)
        em.record()
        rep = ei.ei_reconstruct(G, s_exp, vol, tol=tol, max_iter=max_iter, raise_on_error=False)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        it = rep.iterations
        out[start] = {"seconds": t, "seconds_per_1024_slice": t / eq,
                      "ms_per_1024_slice": 1e3 * t / eq,
                      "start_seconds": e0.elapsed_time(em) * 1e-3,
                      "iterations_mean": float(it.mean()),
                      "iterations_median": float(np.median(it)), "iterations_max": int(it.max()),
                      "projections_per_iteration": float(rep.slice_projections.sum()) /
                      max(1, int(it.sum())),
                      "converged": int(rep.converged.sum()), "slices": int(len(it)),
                      "f_final": rep.f_final.tolist()}
        del vol
    if "zero" in out:
        zf = np.asarray(out["zero"]["f_final"])
        for k in out:
            if k != "zero":
                out[k]["f_final_rel_diff_vs_zero_max"] = float(
                    np.max(np.abs(np.asarray(out[k]["f_final"]) - zf) / np.abs(zf)))
    for k in out:
        out[k]["f_final_sum"] = float(np.sum(out[k].pop("f_final")))
    return out


def evaluate(net: WarmStartNet, shapes: Sequence[Tuple[int, int, int]], seed0: int, n_m: int = 7,
             tol: float = 1e-6, max_iter: int = 400, max_chunk_voxels: int = 64 * 256 * 256,
             device="cuda"):
    """time_to_tolerance of held-out slices (seeds seed0 + i) in chunks, summed."""
    tot: Dict[str, dict] = {}
    i = 0
    while i < len(shapes):
        j, vox = i, 0
        while j < len(shapes) and (j == i or vox + shapes[j][0] ** 2 <= max_chunk_voxels):
            vox += shapes[j][0] ** 2
            j += 1
        chunk = list(shapes[i:j])
        G, s_exp = synth.build_problem(chunk, n_m, [seed0 + k for k in range(i, j)], device,
                                       seed0 + i)
        r = time_to_tolerance(G, s_exp, ["zero", "single_shot", "cnn"], tol, max_iter, net)
        w = j - i
        for k, v in r.items():
            t = tot.setdefault(k, {"seconds": 0.0, "slices": 0, "converged": 0, "iter_sum": 0.0,
                                   "iterations_max": 0, "f_final_sum": 0.0,
                                   "f_final_rel_diff_vs_zero_max": 0.0})
            t["seconds"] += v["seconds"]
            t["slices"] += v["slices"]
            t["converged"] += v["converged"]
            t["iter_sum"] += v["iterations_mean"] * w
            t["iterations_max"] = max(t["iterations_max"], v["iterations_max"])
            t["f_final_sum"] += v["f_final_sum"]
            t["f_final_rel_diff_vs_zero_max"] = max(t["f_final_rel_diff_vs_zero_max"],
                                                    v.get("f_final_rel_diff_vs_zero_max", 0.0))
        G.close()
        i = j
    eq = sum(n * n for n, _, _ in shapes) / 1024.0 ** 2
    for k, t in tot.items():
        t["iterations_mean"] = t.pop("iter_sum") / t["slices"]
        t["seconds_per_1024_slice"] = t["seconds"] / eq
    return tot


# ------------------------------------------------------------------ command line
def shapes_for(name: str, count: int, seed: int) -> List[Tuple[int, int, int]]:
    """Slice shapes: "256" = 256x256, 720 angles, 384 pixels; "uneven1024" =
    the uneven 1024/512 batch's shapes (1800 angles, detector pixels drawn as in
    that workload, with `seed` for the draw)."""
    from . import workloads
    if name == "256":
        return [(256, 720, 384)] * count
    if name == "uneven1024":
        sl = workloads.uneven1024(seed=seed).slices
        return [sl[i % len(sl)] for i in range(count)]
    raise ValueError(name)


def main(argv: Sequence[str] | None = None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", default="256", choices=["256", "uneven1024"])
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--eval", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--steps-per-epoch", type=int, default=None)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--crop", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    pairs, it = generate_pairs(shapes_for(args.shapes, args.pairs, 6), 1_000_000)
    torch.cuda.synchronize()
    t1 = time.time()
    net = WarmStartNet(levels=args.levels, base=args.base, crop=args.crop, batch=args.batch)
    hist = train(net, pairs, args.epochs, args.lr, lr_final=args.lr * 0.05,
                 steps_per_epoch=args.steps_per_epoch)
    torch.cuda.synchronize()
    t2 = time.time()
    if args.save:
        net.save(args.save)
    del pairs
    ev = evaluate(net, shapes_for(args.shapes, args.eval, 5), 2_000_000)
    print(json.dumps({"shapes": args.shapes, "pairs": args.pairs, "pair_generation_s": t1 - t0,
                      "training_s": t2 - t1, "pair_iterations_mean": float(it.mean()),
                      "loss_per_epoch": hist, "eval": ev}))


if __name__ == "__main__":
    main()
