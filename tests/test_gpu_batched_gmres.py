"""GPU parity of the batched persistent GMRES(m) (GS(p) + GMRES(m) with CGS2,
one block per system) against the oracle, through the C ABI; the launch
shapes (block size 128 / 256 / 512) and the routing of large systems to the
grid-wide solvers, for both batched solvers."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import gsk
from problems import cd, configs

pytestmark = pytest.mark.gpu


def _upload(g, systems):
    import torch

    As = [g.Csr.from_host(s.rowptr, s.colidx, s.val) for s in systems]
    bs = [torch.as_tensor(s.b, device="cuda") for s in systems]
    xs = [torch.zeros(s.n, dtype=torch.float64, device="cuda") for s in systems]
    return As, bs, xs


def _gs(s, p):
    if p != p:
        return s
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, p)
    return cd.System(s.n, s.rowptr, s.colidx, val, b, s.x_true)


def _ensemble(sc, m, tol, maxit, size=8):
    """The oracle on b and on size-1 copies of b perturbed by <= 1 ulp: on
    these inclusion systems restarted GMRES can sit near stagnation, and its
    step count then moves a lot under rounding (the parity bar of the
    single-system tests)."""
    out = [oracle.gmres(sc.rowptr, sc.colidx, sc.val, sc.b, m=m, tol=tol, maxit=maxit)[1]]
    for seed in range(1, size):
        u = np.random.default_rng(seed).uniform(-1.0, 1.0, sc.n)
        out.append(oracle.gmres(sc.rowptr, sc.colidx, sc.val, sc.b * (1.0 + u * np.finfo(np.float64).eps), m=m,
                                tol=tol, maxit=maxit)[1])
    return out


def _parity_batch():
    """Systems of several kinds, sizes, scalings and restart lengths: ones on
    which GMRES(m) converges (counts checked against the oracle's rounding
    ensemble) and two inclusion systems on which it stagnates (both sides
    stop at maxit with comparable metrics)."""
    cases = [(configs.c4_system(1), 1.0, 13), (configs.c4_system(10), math.inf, 19),
             (configs.c4_system(14), math.inf, 10), (configs.c1(), 2.0, 20), (configs.c2(12), 2.0, 30),
             (configs.p1(32), 2.0, 10), (configs.c1(24), float("nan"), 25),
             (configs.c4_system(2), math.inf, 16)]
    return [c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases]


def test_batched_gmres_matches_oracle():
    g = gsk()
    systems, ps, ms = _parity_batch()
    maxit = 1000
    As, bs, xs = _upload(g, systems)
    infos, stat = g.gmres_solve_batched(As, bs, xs, m=ms, p=ps, tol=1e-8, options=g.opts(maxit=maxit))
    assert all(st == g.OK for st in stat)
    seen = set()
    for s, m, p, x, info in zip(systems, ms, ps, xs, infos):
        sc = _gs(s, p)
        xg = x.cpu().numpy()
        mu = oracle.relres(sc.rowptr, sc.colidx, sc.val, sc.b, xg)
        assert abs(mu - info["relres_true"]) <= 1e-6 * mu + 1e-15, (mu, info)
        _, io = oracle.gmres(sc.rowptr, sc.colidx, sc.val, sc.b, m=m, tol=1e-8, maxit=maxit)
        seen.add(io["conv"])
        if io["conv"] == oracle.CONVERGED:
            assert info["conv"] == 0 and mu < 1e-8, (info, io)
            ens = [io] + _ensemble(sc, m, 1e-8, maxit, size=4)[1:]
            its = [e["iters"] for e in ens]
            lo, hi = min(its), max(its)
            assert min(0.95 * lo, lo - 2) <= info["iters"] <= max(1.05 * hi, hi + 2), (p, m, info, its)
        else:
            assert info["conv"] == io["conv"], (info, io)
            assert mu <= 10 * io["relres_true"] and io["relres_true"] <= 10 * mu, (mu, io)
    assert seen == {oracle.CONVERGED, oracle.MAXIT}


def test_batched_gmres_same_alone_and_in_the_batch():
    import torch

    g = gsk()
    systems = [configs.c4_system(i) for i in range(10)]
    As, bs, xs = _upload(g, systems)
    g.gmres_solve_batched(As, bs, xs, m=20, p=2.0, tol=1e-8)
    for k in (3, 7):
        A1, b1, x1 = _upload(g, [systems[k]])
        g.gmres_solve_batched(A1, b1, x1, m=20, p=2.0, tol=1e-8)
        assert torch.equal(x1[0], xs[k])


@pytest.mark.parametrize("block", [128, 256, 512])
@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_batched_block_sizes(block, solver):
    g = gsk()
    systems = [configs.c4_system(i) for i in range(12)]
    As, bs, xs = _upload(g, systems)
    o = g.opts(batch_block=block)
    if solver == "gmres":
        infos, stat = g.gmres_solve_batched(As, bs, xs, m=20, p=2.0, tol=1e-8, options=o)
    else:
        infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=o)
    assert all(st == g.OK for st in stat)
    for s, x, info in zip(systems, xs, infos):
        sc = _gs(s, 2.0)
        if info["conv"] == 0:
            assert oracle.relres(sc.rowptr, sc.colidx, sc.val, sc.b, x.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_large_systems_take_the_grid_wide_solver(solver):
    """With batch_large_n, the systems above it are solved by gs_scale and the
    single-system solver: bit-identical to those calls made directly."""
    import torch

    g = gsk()
    systems = [configs.c4_system(i) for i in range(8)]
    big = max(s.n for s in systems)
    thr = sorted(s.n for s in systems)[4]
    As, bs, xs = _upload(g, systems)
    o = g.opts(batch_large_n=thr)
    if solver == "gmres":
        infos, stat = g.gmres_solve_batched(As, bs, xs, m=20, p=2.0, tol=1e-8, options=o)
    else:
        infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=o)
    assert all(st == g.OK for st in stat)
    for s, x, info in zip(systems, xs, infos):
        if s.n > thr:
            A1, b1, x1 = _upload(g, [s])
            g.gs_scale(A1[0], b1[0], p=2.0)
            ref = (g.gmres_solve(A1[0], b1[0], x1[0], m=20, tol=1e-8) if solver == "gmres"
                   else g.bicgstab_solve(A1[0], b1[0], x1[0], tol=1e-8))
            assert torch.equal(x1[0], x) and ref["iters"] == info["iters"]
    assert big > thr


def test_routed_systems_run_beside_the_batch():
    """The systems above batch_large_n run on the grid-wide lane beside the
    persistent launch (a second stream, a child context): the batch's own
    systems give bitwise the results of a batch without them, the routed ones
    those of direct calls, and a failing routed system reports its own
    status (and its error text) while the others complete."""
    import torch

    g = gsk()
    systems = [configs.c4_system(i) for i in range(10)]
    thr = sorted(s.n for s in systems)[5]
    As, bs, xs = _upload(g, systems)
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=g.opts(batch_large_n=thr))
    assert all(st == g.OK for st in stat)
    small = [i for i, s in enumerate(systems) if s.n <= thr]
    large = [i for i, s in enumerate(systems) if s.n > thr]
    assert small and large
    A2, b2, x2 = _upload(g, [systems[i] for i in small])
    inf2, _ = g.bicgstab_solve_batched(A2, b2, x2, p=2.0, tol=1e-8)
    for q, i in enumerate(small):
        assert torch.equal(x2[q], xs[i]) and inf2[q]["iters"] == infos[i]["iters"]
    for i in large:
        A1, b1, x1 = _upload(g, [systems[i]])
        g.gs_scale(A1[0], b1[0], p=2.0)
        ref = g.bicgstab_solve(A1[0], b1[0], x1[0], tol=1e-8)
        assert torch.equal(x1[0], xs[i]) and ref["iters"] == infos[i]["iters"]
    # a routed system with a zero row
    bad = large[0]
    s = systems[bad]
    val = s.val.copy()
    val[s.rowptr[3]:s.rowptr[4]] = 0.0
    systems_bad = list(systems)
    systems_bad[bad] = cd.System(s.n, s.rowptr, s.colidx, val, s.b)
    As, bs, xs = _upload(g, systems_bad)
    with pytest.raises(g.GskError) as ei:
        g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=g.opts(batch_large_n=thr))
    assert ei.value.status == g.ERR_ZERO_ROW
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=g.opts(batch_large_n=thr),
                                           check=False)
    assert stat[bad] == g.ERR_ZERO_ROW
    assert all(st == g.OK for i, st in enumerate(stat) if i != bad)


def test_batched_gmres_rejects_bad_shapes():
    g = gsk()
    systems = [configs.c4_system(0)]
    As, bs, xs = _upload(g, systems)
    for o in (g.opts(batch_block=100), g.opts(precision=g.PREC_MIXED)):
        with pytest.raises(g.GskError) as e:
            g.gmres_solve_batched(As, bs, xs, m=20, p=2.0, tol=1e-8, options=o)
        assert e.value.status == g.ERR_ARG
    with pytest.raises(g.GskError):
        g.gmres_solve_batched(As, bs, xs, m=65, p=2.0, tol=1e-8)


def _well_conditioned(seed, n):
    rs = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        c = np.unique(np.concatenate([[i], rs.integers(0, n, 6)]))
        v = rs.uniform(-1, 1, len(c))
        v[c == i] = rs.uniform(2, 3) * 7
        rows.append(len(c))
        cols.append(c)
        vals.append(v)
    rp = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
    return cd.System(n, rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals), rs.normal(size=n))


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_batched_counts_match_the_oracle_exactly_where_rounding_does_not_matter(solver):
    """Well-conditioned nonsymmetric systems of several sizes, no scaling:
    each system takes exactly the oracle's iterations (block-level sums in
    another order do not move the count there) and reaches its solution."""
    g = gsk()
    systems = [_well_conditioned(s, n) for s, n in ((1, 300), (2, 1500), (3, 4000), (4, 777))]
    As, bs, xs = _upload(g, systems)
    o = g.opts(metric=g.METRIC_PLAIN, refresh=0)
    nan = float("nan")
    if solver == "gmres":
        infos, stat = g.gmres_solve_batched(As, bs, xs, m=10, p=[nan] * 4, tol=1e-10, options=o)
    else:
        infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=[nan] * 4, tol=1e-10, options=o)
    assert all(st == g.OK for st in stat)
    for s, x, info in zip(systems, xs, infos):
        if solver == "gmres":
            xo, io = oracle.gmres(s.rowptr, s.colidx, s.val, s.b, m=10, tol=1e-10, w=np.ones(s.n))
        else:
            xo, io = oracle.bicgstab(s.rowptr, s.colidx, s.val, s.b, tol=1e-10, refresh=0, w=np.ones(s.n))
        assert info["conv"] == io["conv"] == 0 and info["iters"] == io["iters"], (s.n, info, io)
        assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()
