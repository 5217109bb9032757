"""The batched solvers' autotuner on the GPU: it times the candidate launch
shapes on a sample of a C4-style batch, returns one of them, caches it, and
the caller's data is untouched by the tuning."""
import time

import pytest

import oracle
from gpu_util import gsk
from problems import configs

pytestmark = pytest.mark.gpu


def test_autotune_batched(tmp_path, monkeypatch):
    import torch

    monkeypatch.setenv("GSK_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    g = gsk()
    from paper_0812_2769_gb300 import autotune

    systems = [configs.c4_system(i) for i in range(48)]
    As = [g.Csr.from_host(s.rowptr, s.colidx, s.val) for s in systems]
    bs = [torch.as_tensor(s.b, device="cuda") for s in systems]
    xs = [torch.zeros(s.n, dtype=torch.float64, device="cuda") for s in systems]
    v0 = [A.val.clone() for A in As]
    cfg = autotune.batched_config(As, bs, xs, solver="bicgstab", p=2.0, sample=24, reps=1)
    assert cfg["batch_block"] in autotune.BLOCKS and cfg["batch_large_n"] >= 0
    assert all(torch.equal(A.val, v) for A, v in zip(As, v0))  # tuning worked on copies
    assert all(torch.count_nonzero(x) == 0 for x in xs)
    t0 = time.perf_counter()
    assert autotune.batched_config(As, bs, xs, solver="bicgstab", p=2.0, sample=24, reps=1) == cfg  # cache hit
    assert time.perf_counter() - t0 < 1.0
    infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8, options=g.opts(**cfg))
    assert all(s == g.OK for s in stat)
    for s, x, info in zip(systems, xs, infos):
        if info["conv"] == 0:
            val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
            assert oracle.relres(s.rowptr, s.colidx, val, b, x.cpu().numpy()) < 1e-8
