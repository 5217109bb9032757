"""The batched solvers' autotuner, host logic (no GPU): the sample spans
the batch's size range, the cache round-trips, the key separates batches
that need separate tuning."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

from paper_0812_2769_gb300 import autotune  # noqa: E402


class _A:
    def __init__(self, n, nnz):
        self.n, self.nnz = n, nnz
        self.val = torch.zeros(1)


def test_sample_spans_the_sizes():
    As = [_A(n, 5 * n) for n in range(100, 1100)]
    idx = autotune._sample_indices(As, 10)
    assert len(idx) == 10 and len(set(idx)) == 10
    ns = sorted(As[i].n for i in idx)
    assert ns[0] == 100 and ns[-1] >= 1000
    assert autotune._sample_indices(As[:5], 10) == sorted(range(5), key=lambda i: As[i].n)


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("GSK_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load(str(path)) == {}
    autotune._store(str(path), {"k": {"batch_block": 128, "batch_large_n": 0}})
    assert json.load(open(path)) == {"k": {"batch_block": 128, "batch_large_n": 0}}
    assert not os.path.exists(str(path) + ".tmp")


def test_key_separates_batches():
    small = [_A(256, 1200)] * 64
    large = [_A(16384, 80000)] * 64
    k1 = autotune.batch_key(small, "bicgstab", 0, 30)
    assert k1 != autotune.batch_key(large, "bicgstab", 0, 30)
    assert k1 != autotune.batch_key(small, "gmres", 0, 30)
    assert k1 != autotune.batch_key(small, "bicgstab", 1, 30)
    assert k1 == autotune.batch_key(list(small), "bicgstab", 0, 30)
