"""Named synthetic workloads.

Every workload is a seeded convection-diffusion system built by
:mod:`problems.cd`.  Random draws come from SplitMix64 (:mod:`problems.rng`)
with fixed seeds, so every consumer of a workload sees identical arrays.

* ``c1``  2D, 32x32 interior, a = 1000 on [1/4, 3/4]^2 else 1, beta = (10, 10),
  x_true ~ U[-1, 1) (seed 0), b = A x_true.  n = 1024.
* ``c2``  3D, 128^3 interior, a on a 4x4x4 checkerboard alternating 1 / 1e4,
  beta = (20, 20, 20), seeded x_true.  n = 2,097,152.
* ``c3``  3D, 256^3, a = 10^U[-3, 3] per cell of an 8^3 partition, beta per
  cell U[-30, 30]^3, seeded x_true.  n = 16,777,216.
* ``c4_system(i)``  one of the 4096 batch systems: side L ~ U{16..128}, a = 1
  with 1..5 circular inclusions (centre U[0.1, 0.9]^2, radius U[0.05, 0.2],
  contrast 10^U[2, 6], overlaps take the max), beta ~ U[-10, 10]^2,
  x_true seed 1000 + i.
* ``p1``  the paper's Problem 1 (Sec. 3): a = b = 10^3 (or 10^4) on the open
  square (1/4, 3/4)^2 else 1, conservative convection d = 10(x+y),
  e = 10(x-y), u = 0 on the boundary, right-hand side b = A (1, ..., 1)^T.
  ``continuous`` gives the variants with a = b constant everywhere.
* ``p4``  the paper's Problem 4 (Sec. 6): 3D, a = D on the open cube
  (1/3, 2/3)^3 else 1, convection d = e = f (default 100), u = 1 on the
  z = 0 face and 0 on the other faces, zero source.

The grid size N is a parameter everywhere so that tests can build small
instances of the same family.
"""
from __future__ import annotations

import numpy as np

from . import cd, rng

SEED_XTRUE = 0
SEED_C3_A = 0x3A
SEED_C3_BETA = 0x3B
SEED_C4_PARAMS = 4_000_000
SEED_C4_XTRUE = 1000


def c1(N: int = 32) -> cd.System:
    s = cd.build(N, 2, cd.InnerBox((1, 4), (3, 4), 1000.0, 1.0), [cd.Constant(10.0)] * 2)
    # closed square [1/4, 3/4]^2: no face of a 32x32 grid lies on its edge
    s = cd.manufacture(s, rng.x_true(SEED_XTRUE, s.n))
    s.meta.update(name=f"c1 2D {N}x{N} inner-square a=1e3, beta=(10,10)")
    return cd.release_slots(s)


def c2(N: int = 128) -> cd.System:
    s = cd.build(N, 3, cd.Checkerboard(4, 1.0, 1.0e4), [cd.Constant(20.0)] * 3)
    s = cd.manufacture(s, rng.x_true(SEED_XTRUE, s.n))
    s.meta.update(name=f"c2 3D {N}^3 checkerboard 4^3 a=1/1e4, beta=(20,20,20)")
    return cd.release_slots(s)


def c3_fields(K: int = 8):
    a = 10.0 ** rng.uniform(SEED_C3_A, K**3, -3.0, 3.0).reshape(K, K, K)
    bt = rng.uniform(SEED_C3_BETA, 3 * K**3, -30.0, 30.0).reshape(3, K, K, K)
    return cd.CellTable(K, a), [cd.CellTable(K, bt[d]) for d in range(3)]


def c3(N: int = 256) -> cd.System:
    a, beta = c3_fields()
    s = cd.build(N, 3, a, beta)
    s = cd.manufacture(s, rng.x_true(SEED_XTRUE, s.n))
    s.meta.update(name=f"c3 3D {N}^3 log-uniform 8^3 partition a=10^U[-3,3], beta=U[-30,30]^3")
    return cd.release_slots(s)


def c4_params(i: int) -> dict:
    """Parameters of batch system i (all from one SplitMix64 stream)."""
    u = rng.uniform01(SEED_C4_PARAMS + i, 32)
    L = 16 + int(u[0] * 113)  # U{16..128}
    k = 1 + int(u[1] * 5)  # U{1..5}
    centres = np.stack([0.1 + 0.8 * u[2 : 2 + k], 0.1 + 0.8 * u[7 : 7 + k]], axis=1)
    radii = 0.05 + 0.15 * u[12 : 12 + k]
    contrasts = 10.0 ** (2.0 + 4.0 * u[17 : 17 + k])
    beta = (-10.0 + 20.0 * u[22], -10.0 + 20.0 * u[23])
    return dict(L=L, k=k, centres=centres, radii=radii, contrasts=contrasts, beta=beta)


def c4_system(i: int) -> cd.System:
    p = c4_params(i)
    a = cd.Inclusions(p["centres"], p["radii"], p["contrasts"])
    s = cd.build(p["L"], 2, a, [cd.Constant(p["beta"][0]), cd.Constant(p["beta"][1])])
    s = cd.manufacture(s, rng.x_true(SEED_C4_XTRUE + i, s.n))
    s.meta.update(name=f"c4[{i}] 2D {p['L']}^2 {p['k']} inclusions", **{"L": p["L"]})
    return cd.release_slots(s)


def c4_sides(count: int = 4096) -> np.ndarray:
    return np.array([c4_params(i)["L"] for i in range(count)])


def p1(N: int = 128, inner: float = 1.0e3, continuous: float | None = None) -> cd.System:
    if continuous is not None:
        a = cd.Constant(continuous)
    else:
        a = cd.InnerBox((1, 4), (3, 4), inner, 1.0)
    beta = [cd.Affine(0.0, (10.0, 10.0)), cd.Affine(0.0, (10.0, -10.0))]
    s = cd.build(N, 2, a, beta, conservative=True)
    s.b = cd.apply(s, np.ones(s.n))
    s.meta.update(name=f"p1 2D {N}x{N}")
    return cd.release_slots(s)


def p4(N: int = 80, D: float = 1.0e4, conv: float = 100.0, continuous: bool = False) -> cd.System:
    a = cd.Constant(D) if continuous else cd.InnerBox((1, 3), (2, 3), D, 1.0)

    def g(axis, side, nums, den):
        # u = 1 on the z = 0 face, 0 on every other face
        return np.asarray(1.0 if (axis == 2 and side == -1) else 0.0)

    s = cd.build(N, 3, a, [cd.Constant(conv)] * 3, dirichlet=g)
    s.meta.update(name=f"p4 3D {N}^3 D={D:g} conv={conv:g}")
    return cd.release_slots(s)
