"""Seeded request streams for the serving workload.

Each request is a convection-diffusion solve: 2D with side log-uniform in
[side2d_min, side2d_max] or 3D with side log-uniform in [side3d_min,
side3d_max] (50/50), a checkerboard or circular-inclusion coefficient field
(50/50) with contrast 10^U[2, 6], a random convection vector, GMRES(m) with
m ~ U{10..50} or Bi-CGSTAB (50/50), and GS(p) with p in {1, 2, inf}.
Arrivals form a Poisson process of rate `rate` (requests per second).
All draws come from SplitMix64 with seed `seed`; nothing here solves anything.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import cd, rng


@dataclass
class RequestSpec:
    rid: int
    arrival: float  # seconds after the stream starts
    dim: int
    side: int
    field: str  # "checkerboard" or "inclusions"
    contrast: float
    solver: str  # "gmres" or "bicgstab"
    m: int
    p: float
    seed: int

    def build(self) -> cd.System:
        u = rng.uniform01(self.seed, 32)
        if self.field == "checkerboard":
            K = 2 + int(u[0] * 7)  # 2..8 cells per axis
            a = cd.Checkerboard(K, 1.0, self.contrast)
        else:
            k = 1 + int(u[1] * 5)
            d = self.dim
            cen = np.stack([0.1 + 0.8 * u[2 + 5 * j: 2 + 5 * j + k] for j in range(d)], axis=1)
            rad = 0.05 + 0.15 * u[17:17 + k]
            a = cd.Inclusions(cen, rad, np.full(k, self.contrast))
        beta = [cd.Constant(-20.0 + 40.0 * u[24 + j]) for j in range(self.dim)]
        s = cd.build(self.side, self.dim, a, beta)
        s = cd.manufacture(s, rng.x_true(self.seed + 1, s.n))
        s.meta.update(name=f"req{self.rid} {self.dim}D {self.side}")
        return cd.release_slots(s)


def stream(count: int, rate: float, seed: int = 7, side2d=(64, 1024), side3d=(16, 160)) -> list[RequestSpec]:
    u = rng.uniform01(seed, 10 * count).reshape(count, 10)
    t = np.cumsum(-np.log1p(-u[:, 0]) / rate)  # exponential inter-arrival times
    out = []
    for i in range(count):
        dim = 2 if u[i, 1] < 0.5 else 3
        lo, hi = side2d if dim == 2 else side3d
        side = int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u[i, 2])))
        out.append(RequestSpec(
            rid=i, arrival=float(t[i]), dim=dim, side=side,
            field="checkerboard" if u[i, 3] < 0.5 else "inclusions",
            contrast=10.0 ** (2.0 + 4.0 * u[i, 4]),
            solver="gmres" if u[i, 5] < 0.5 else "bicgstab",
            m=10 + int(u[i, 6] * 41),
            p=[1.0, 2.0, math.inf][min(2, int(u[i, 7] * 3))],
            seed=int(seed * 1_000_003 + 17 * i)))
    return out
