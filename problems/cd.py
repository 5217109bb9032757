"""Seeded convection-diffusion test systems in CSR form.

The operator is  -div(a grad u) + beta . grad u  (or the conservative
convection div(beta u) of Problem 1) on the unit square or cube with Dirichlet
boundary values, discretised on N interior points per axis (h = 1/(N+1)) with
the three-point central formula of Sec. 2.1: the diffusion flux through each
face uses the coefficient at the face midpoint, a_{i+1/2}.  Every row is
multiplied by h^2, so a row carries O(a) entries: the diagonal is the sum of
the face coefficients and the convection contributes +-h*beta/2 to the
neighbours (the paper's eigenvalue tables, Table 1b / 4a, show entries of
this size).  Points outside the domain are eliminated; their Dirichlet value
moves to the right-hand side.

Rows are numbered lexicographically with x fastest; each row's columns are in
ascending order (-z, -y, -x, diagonal, +x, +y, +z).  Indices are int32.

Coordinates are handled as exact rationals num/den with den = 2(N+1) (a node
at index i has num = 2(i+1); its faces num +- 1), so a coefficient field that
is constant on cells [k/K, (k+1)/K) decides a face lying exactly on a cell
boundary by integer arithmetic: such a face belongs to the upper cell.

This module only builds inputs.  It computes no part of the solver method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np


# ----------------------------------------------------------------- fields
class Field:
    """A scalar coefficient as a function of rational coordinates."""

    def __call__(self, nums: Sequence[np.ndarray], den: int) -> np.ndarray:  # pragma: no cover
        raise NotImplementedError


@dataclass
class Constant(Field):
    value: float

    def __call__(self, nums, den):
        shape = np.broadcast_shapes(*[np.shape(c) for c in nums])
        return np.full(shape, float(self.value))


@dataclass
class InnerBox(Field):
    """``inside`` where lo < x_d < hi for every axis d (strict), else ``outside``.
    lo and hi are given as fractions (p, q)."""

    lo: tuple
    hi: tuple
    inside: float
    outside: float

    def __call__(self, nums, den):
        (lp, lq), (hp, hq) = self.lo, self.hi
        inside = None
        for c in nums:
            c = np.asarray(c, dtype=np.int64)
            m = (c * lq > lp * den) & (c * hq < hp * den)
            inside = m if inside is None else (inside & m)
        return np.where(inside, float(self.inside), float(self.outside))


def _cells(nums, den, K):
    return [np.minimum((np.asarray(c, dtype=np.int64) * K) // den, K - 1) for c in nums]


@dataclass
class Checkerboard(Field):
    """K^d checkerboard of half-open cells: ``even`` where the sum of the cell
    indices is even, else ``odd``."""

    K: int
    even: float
    odd: float

    def __call__(self, nums, den):
        s = sum(_cells(nums, den, self.K))
        return np.where(s % 2 == 0, float(self.even), float(self.odd))


@dataclass
class CellTable(Field):
    """Piecewise constant on the K^d partition; ``table`` is indexed [cx, cy(, cz)]."""

    K: int
    table: np.ndarray

    def __call__(self, nums, den):
        idx = _cells(nums, den, self.K)
        return self.table[tuple(idx)]


@dataclass
class Inclusions(Field):
    """Background 1 with circular (spherical) inclusions; where inclusions
    overlap the largest contrast wins.  Points strictly inside count."""

    centres: np.ndarray  # [k, d]
    radii: np.ndarray  # [k]
    contrasts: np.ndarray  # [k]
    background: float = 1.0

    def __call__(self, nums, den):
        xs = [np.asarray(c, dtype=np.float64) / den for c in nums]
        shape = np.broadcast_shapes(*[np.shape(c) for c in xs])
        out = np.full(shape, float(self.background))
        for cen, r, con in zip(self.centres, self.radii, self.contrasts):
            d2 = sum((x - c) ** 2 for x, c in zip(xs, cen))
            out = np.where(d2 < r * r, np.maximum(out, con), out)
        return out


@dataclass
class Affine(Field):
    """c0 + sum_d coef[d] * x_d (Problem 1's d = 10(x+y), e = 10(x-y))."""

    c0: float
    coef: tuple

    def __call__(self, nums, den):
        out = float(self.c0)
        for c, k in zip(nums, self.coef):
            out = out + float(k) * (np.asarray(c, dtype=np.float64) / den)
        shape = np.broadcast_shapes(*[np.shape(c) for c in nums])
        return np.broadcast_to(np.asarray(out, dtype=np.float64), shape)


# ----------------------------------------------------------------- system
@dataclass
class System:
    """A sparse linear system A x = b in CSR form (host numpy arrays)."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    b: np.ndarray  # float64 [n]
    x_true: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        A[rows, self.colidx] = self.val
        return A


def _axes_nums(N: int, dim: int):
    """Node numerators 2(i+1) as broadcastable arrays, axis order (x, y, z)
    with x varying fastest in the flattened (C-order) array."""
    base = 2 * (np.arange(N, dtype=np.int64) + 1)
    nums = []
    for d in range(dim):
        shape = [1] * dim
        shape[dim - 1 - d] = N  # x is the last (fastest) array axis
        nums.append(base.reshape(shape))
    return nums


def build(
    N: int,
    dim: int,
    a: Field,
    beta: Sequence[Field],
    conservative: bool = False,
    dirichlet: Callable | None = None,
) -> System:
    """Assemble the h^2-scaled central-difference system (see module doc).

    ``beta[d]`` is the convection component along axis d.  Non-conservative
    convection beta . grad u is evaluated at the row's node; the conservative
    form div(beta u) evaluates beta at the neighbour node (Problem 1).
    ``dirichlet(axis, side, nums, den)`` gives the boundary value for the
    neighbour eliminated on that side (default 0); it returns an array
    broadcastable to the grid.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    den = 2 * (N + 1)
    h = 1.0 / (N + 1)
    shape = (N,) * dim
    n = N**dim
    nums = _axes_nums(N, dim)
    full = lambda arr: np.broadcast_to(arr, shape)

    node_index = np.arange(n, dtype=np.int64).reshape(shape)
    strides = [N**d for d in range(dim)]  # x stride 1, y stride N, z stride N^2

    nslot = 2 * dim + 1
    val = np.zeros((n, nslot))
    col = np.zeros((n, nslot), dtype=np.int64)
    mask = np.zeros((n, nslot), dtype=bool)
    diag = np.zeros(shape)
    rhs = np.zeros(shape)

    beta_node = [full(bf(nums, den)) for bf in beta] if not conservative else None

    # slot order: -z, -y, -x, diag, +x, +y, +z  (2D: -y, -x, diag, +x, +y)
    for d in range(dim):
        for side in (-1, +1):
            slot = dim + side * (d + 1)
            fnums = list(nums)
            fnums[d] = nums[d] + side  # face midpoint numerator
            a_face = full(a(fnums, den))
            diag += a_face
            if conservative:
                nnums = list(nums)
                nnums[d] = nums[d] + 2 * side
                conv = side * 0.5 * h * full(beta[d](nnums, den))
            else:
                conv = side * 0.5 * h * beta_node[d]
            coef = -a_face + conv
            # index of the node along axis d, broadcast to the grid
            idx_d = full((nums[d] // 2) - 1)
            inside = (idx_d + side >= 0) & (idx_d + side < N)
            val[:, slot] = np.where(inside, coef, 0.0).reshape(-1)
            col[:, slot] = (node_index + side * strides[d]).reshape(-1)
            mask[:, slot] = inside.reshape(-1)
            if dirichlet is not None:
                bnums = list(nums)
                bnums[d] = nums[d] + 2 * side
                g = full(dirichlet(d, side, bnums, den))
                rhs -= np.where(inside, 0.0, coef * g)
    val[:, dim] = diag.reshape(-1)
    col[:, dim] = node_index.reshape(-1)
    mask[:, dim] = True

    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    sys_ = System(
        n=n,
        rowptr=rowptr.astype(np.int32),
        colidx=col[mask].astype(np.int32),
        val=val[mask],
        b=rhs.reshape(-1).copy(),
        meta={"N": N, "dim": dim, "h": h},
    )
    sys_._slots = (val, col, mask)  # kept for the manufactured right-hand side
    return sys_


def apply(sys_: System, x: np.ndarray) -> np.ndarray:
    """A x for building a manufactured right-hand side (input generation only)."""
    slots = getattr(sys_, "_slots", None)
    if slots is not None:
        val, col, mask = slots
        return np.where(mask, val * x[np.where(mask, col, 0)], 0.0).sum(axis=1)
    out = np.zeros(sys_.n)
    rows = np.repeat(np.arange(sys_.n), np.diff(sys_.rowptr))
    np.add.at(out, rows, sys_.val * x[sys_.colidx])
    return out


def manufacture(sys_: System, x_true: np.ndarray) -> System:
    """Set b = A x_true and remember x_true."""
    sys_.b = apply(sys_, x_true)
    sys_.x_true = x_true
    return sys_


def release_slots(sys_: System) -> System:
    """Drop the dense [n, 2d+1] assembly arrays once b is built."""
    if hasattr(sys_, "_slots"):
        del sys_._slots
    return sys_
