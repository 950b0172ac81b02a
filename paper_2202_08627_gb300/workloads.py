"""Synthetic workloads shaped like the paper's scans (sizes and seeds only).

Every slice has the field of view inputs.FOV_CM, angles theta_a = a pi / n_theta,
mask positions inputs.mask_positions(M), a seeded 8-ellipse phantom and a
seeded per-pixel Gaussian flat IC.  The measured ICs are the IC model applied
to the phantom's exact line integrals, plus Poisson noise at 1e4 counts.

  small        one 64x64 slice, 90 angles, 96 pixels, M = 7 (20 L-BFGS iterations)
  batch256     64 slices of 256x256, 720 angles, 384 pixels, M = 7
  check128     one 128x128 slice, 180 angles, 192 pixels, M = 5
  uneven1024   256 slices, half 1024x1024 and half 512x512 (interleaved), 1800
               angles, detector pixels drawn per slice from {1024, 1152, 1280,
               1408, 1536}, M = 7 (about 16.5 GB of measured ICs)
  pure1024     the 128 slices of 1024x1024 of uneven1024
  single1024   one 1024x1024 slice of that shape (1800 angles, 1536 pixels,
               M = 7)
  batch8x1024  eight such slices: the case the kernel profiles are captured on
               (134 MB volume, 620 MB of measured ICs: larger than L2, a few GB
               on the device in all)
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from . import inputs


@dataclass
class Workload:
    name: str
    description: str
    slices: List[Tuple[int, int, int]]     # (n, n_theta, n_det) per slice
    n_m: int
    seed0: int = 0

    @property
    def n_slices(self) -> int:
        return len(self.slices)

    def per_slice(self):
        return [(n, nth, nd, inputs.pitch_for(n)) for (n, nth, nd) in self.slices]

    # algorithmic bytes of one objective+gradient evaluation: what each kernel
    # must read and write once, whatever its traffic through the caches:
    #   projector 16 n^2 + 12 n_theta n_det, adjoint 32 n^2 + 16 n_theta n_det,
    #   IC kernel (12 + 4 M + 16) n_theta n_det
    def fwd_bytes(self) -> int:
        return sum(16 * n * n + 12 * nth * nd for (n, nth, nd) in self.slices)

    def adj_bytes(self) -> int:
        return sum(32 * n * n + 16 * nth * nd for (n, nth, nd) in self.slices)

    def ic_bytes(self) -> int:
        return sum((28 + 4 * self.n_m) * nth * nd for (n, nth, nd) in self.slices)

    def taps(self) -> int:
        """Matrix entries visited by one projection of the three channels (2 per voxel and angle)."""
        return sum(2 * n * n * nth for (n, nth, nd) in self.slices)

    def voxel_equiv_1024(self) -> float:
        return sum(n * n for (n, _, _) in self.slices) / 1024.0 ** 2

    def meas_bytes(self) -> int:
        return sum(4 * self.n_m * nth * inputs.round_up4(nd) for (n, nth, nd) in self.slices)


def small() -> Workload:
    return Workload("small", "one 64x64 slice, 90 angles, 96 pixels, M=7", [(64, 90, 96)], 7)


def batch256() -> Workload:
    return Workload("batch256", "64 slices of 256x256, 720 angles, 384 pixels, M=7",
                    [(256, 720, 384)] * 64, 7)


def check128() -> Workload:
    return Workload("check128", "one 128x128 slice, 180 angles, 192 pixels, M=5",
                    [(128, 180, 192)], 5)


def uneven1024(seed: int = 5) -> Workload:
    rng = np.random.Generator(np.random.PCG64([seed, 77]))
    dets = rng.choice([1024, 1152, 1280, 1408, 1536], size=256)
    slices = [(1024 if s % 2 == 0 else 512, 1800, int(dets[s])) for s in range(256)]
    return Workload("uneven1024",
                    "256 slices, 50/50 1024x1024 and 512x512 interleaved, 1800 angles, "
                    "1024-1536 detector pixels per slice, M=7", slices, 7)


def pure1024(seed: int = 5) -> Workload:
    """The 1024x1024 half of uneven1024 (same seeds for the detector widths)."""
    sl = [s for s in uneven1024(seed).slices if s[0] == 1024]
    return Workload("pure1024", "the 128 slices of 1024x1024 of the uneven batch, 1800 angles, "
                    "1024-1536 detector pixels per slice, M=7", sl, 7)


def single1024() -> Workload:
    return Workload("single1024", "one 1024x1024 slice, 1800 angles, 1536 pixels, M=7",
                    [(1024, 1800, 1536)], 7)


def batch8x1024() -> Workload:
    return Workload("batch8x1024", "8 slices of 1024x1024, 1800 angles, 1536 pixels, M=7",
                    [(1024, 1800, 1536)] * 8, 7)


WORKLOADS = {"small": small, "batch256": batch256, "check128": check128,
             "uneven1024": uneven1024, "pure1024": pure1024, "single1024": single1024,
             "batch8x1024": batch8x1024}


def shard_slices(slices: List[Tuple[int, int, int]], world: int) -> List[List[int]]:
    """Partition slice indices over `world` ranks, balancing the cost of one
    evaluation (n^2 n_theta voxel-angles + n_theta n_det pixels): longest
    first, each to the least-loaded rank (ties to the lower rank).  Slices are
    independent problems, so the ranks never exchange data while solving."""
    cost = [(n * n * nth + nth * nd, i) for i, (n, nth, nd) in enumerate(slices)]
    cost.sort(key=lambda c: (-c[0], c[1]))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for c, i in cost:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += c
    return [sorted(p) for p in parts]
