"""GPU parity of the batched persistent solver (GS(p) + Bi-CGSTAB, FP64 and
FP32-inner/FP64-refined) against the oracle, through the C ABI."""
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
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, p)
    return cd.System(s.n, s.rowptr, s.colidx, val, b, s.x_true)


def _batch(n=24):
    return [configs.c4_system(i) for i in range(n)]


def test_batched_fp64_matches_oracle_metric_and_scaling():
    g = gsk()
    systems = _batch()
    As, bs, xs = _upload(g, systems)
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8)
    assert all(st == g.OK for st in stat)
    for s, A, b, x, info in zip(systems, As, bs, xs, infos):
        # the batch applied GS(2) in place exactly as the oracle does
        sc = _gs(s, 2.0)
        assert np.allclose(A.val.cpu().numpy(), sc.val, rtol=1e-14, atol=0)
        assert np.allclose(b.cpu().numpy(), sc.b, rtol=1e-14, atol=1e-300)
        xg = x.cpu().numpy()
        mu = oracle.relres(sc.rowptr, sc.colidx, sc.val, sc.b, xg)
        _, io = oracle.bicgstab(sc.rowptr, sc.colidx, sc.val, sc.b, tol=1e-8)
        assert info["conv"] == io["conv"], (info, io)
        if io["conv"] == oracle.CONVERGED:
            assert mu < 1e-8 and abs(mu - info["relres_true"]) <= 1e-6 * mu, (mu, info)
            if s.n <= 2500:  # forward error within cond(A) * tol of x_true
                kappa = np.linalg.cond(sc.dense())
                assert np.linalg.norm(xg - s.x_true) / np.linalg.norm(s.x_true) <= 2 * kappa * 1e-8


def test_batched_iteration_counts_within_oracle_ensemble():
    g = gsk()
    systems = _batch(6)
    As, bs, xs = _upload(g, systems)
    infos, _ = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8)
    for s, info in zip(systems, infos):
        sc = _gs(s, 2.0)
        # the GPU's GS(2) values differ from the oracle's by a few ulp (it
        # multiplies by a reciprocal, the oracle divides), so the ensemble
        # perturbs the scaled values (<= 2 ulp) as well as b (<= 1 ulp); on
        # these inclusion systems the count spreads by up to 30% under such
        # perturbations, so the ensemble is large enough to reach its tails
        its = []
        for seed in range(48):
            rs = np.random.default_rng(seed)
            bb = sc.b if seed == 0 else sc.b * (1 + rs.uniform(-1, 1, s.n) * 2.2e-16)
            vv = sc.val if seed == 0 else sc.val * (1 + rs.uniform(-2, 2, len(sc.val)) * 2.2e-16)
            its.append(oracle.bicgstab(sc.rowptr, sc.colidx, vv, bb, tol=1e-8)[1]["iters"])
        lo, hi = min(its), max(its)
        assert min(0.95 * lo, lo - 2) <= info["iters"] <= max(1.05 * hi, hi + 2), (info["iters"], its)


def test_batched_alone_equals_in_the_mix_bitwise():
    g = gsk()
    systems = _batch(16)
    As, bs, xs = _upload(g, systems)
    g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8)
    for k in (0, 7, 15):
        A1, b1, x1 = _upload(g, [systems[k]])
        g.bicgstab_solve_batched(A1, b1, x1, p=2.0, tol=1e-8)
        assert np.array_equal(x1[0].cpu().numpy(), xs[k].cpu().numpy())


@pytest.mark.parametrize("p", [1.0, math.inf])
def test_batched_other_scalings_use_the_gs2_metric(p):
    g = gsk()
    systems = _batch(8)
    As, bs, xs = _upload(g, systems)
    infos, _ = g.bicgstab_solve_batched(As, bs, xs, p=p, tol=1e-8)
    for s, x, info in zip(systems, xs, infos):
        sp = _gs(s, p)
        _, io = oracle.bicgstab(sp.rowptr, sp.colidx, sp.val, sp.b, tol=1e-8)
        assert info["conv"] == io["conv"], (info, io)
        if info["conv"] == g.CONVERGED:
            sc = _gs(s, 2.0)  # the GS(2)-scaled system defines the metric (Sec. 2.2)
            assert oracle.relres(sc.rowptr, sc.colidx, sc.val, sc.b, x.cpu().numpy()) < 1e-8


def test_batched_unscaled_does_not_converge_like_the_oracle():
    """Without GS the high-contrast batch systems stall in FP64 Bi-CGSTAB, as in
    the oracle (the paper's "no conv." rows); with GS(2) they converge."""
    g = gsk()
    systems = _batch(3)
    As, bs, xs = _upload(g, systems)
    infos, _ = g.bicgstab_solve_batched(As, bs, xs, p=float("nan"), tol=1e-8, options=g.opts(maxit=1500))
    for s, info in zip(systems, infos):
        _, io = oracle.bicgstab(s.rowptr, s.colidx, s.val, s.b, tol=1e-8, maxit=1500)
        assert info["conv"] == io["conv"] == oracle.MAXIT, (info, io)


def test_batched_mixed_precision_refined():
    g = gsk()
    systems = _batch(24)
    As, bs, xs = _upload(g, systems)
    # the batch configuration's tolerance (1e-8) for both precisions
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8,
                                           options=g.opts(precision=g.PREC_MIXED, inner_tol=1e-4))
    for s, x, info in zip(systems, xs, infos):
        assert info["conv"] == g.CONVERGED, info  # the FP64 oracle converges on all 24
        assert info["refinements"] >= 1
        sc = _gs(s, 2.0)
        mu = oracle.relres(sc.rowptr, sc.colidx, sc.val, sc.b, x.cpu().numpy())
        assert mu < 1e-8 and abs(mu - info["relres_true"]) <= 1e-6 * mu


def test_batched_bad_system_is_isolated():
    g = gsk()
    systems = _batch(5)
    bad = systems[2]
    val = bad.val.copy()
    val[bad.rowptr[3]:bad.rowptr[4]] = 0.0
    systems[2] = cd.System(bad.n, bad.rowptr, bad.colidx, val, bad.b, bad.x_true)
    As, bs, xs = _upload(g, systems)
    before = As[2].val.clone()
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, check=False)
    assert stat[2] == g.ERR_ZERO_ROW and As[2].val.equal(before)
    assert all(stat[i] == g.OK and infos[i]["conv"] == g.CONVERGED for i in (0, 1, 3, 4))
