"""Host-side pieces of the benchmark: the algorithmic cost table covers every
kernel the library's profiler reports, its byte and flop counts follow the
operations' definitions, and the recorded DRAM traffic is only used while
it was taken on the current kernel sources."""
import pytest

import bench


def _names():
    from paper_0812_2769_gb300 import lib

    out, k = [], 0
    while True:
        nm = lib().gsk_kernel_name(k).decode()
        if not nm:
            return out
        out.append(nm)
        k += 1


def test_every_profiled_kernel_has_a_cost():
    names = _names()
    assert len(names) >= 18
    for nm in names:
        by, fl = bench.kernel_cost(nm, 3, 1000, 7000)
        assert by > 0, nm


@pytest.mark.parametrize("n,nnz", [(2097152, 14581760), (1024, 4992)])
def test_cost_formulas(n, nnz):
    V = 8 * n
    spmv = 12 * nnz + 4 * (n + 1)
    # the product reads values, indices, row pointers and x once and writes w
    assert bench.kernel_cost("gm_ga_spmv", 0, n, nnz) == (spmv + 2 * V, 2 * nnz + n)
    # CGS passes at step j (k = j + 1 basis columns): pass 1 reads k columns
    # and w; pass 2 reads them and writes w, 2k FMAs per row; pass 3 likewise
    # with k FMAs and the norm
    for j in (0, 14, 29):
        k = j + 1
        assert bench.kernel_cost("gm_gd_cgs_pass1", j, n, nnz) == ((k + 1) * V, 2 * k * n)
        assert bench.kernel_cost("gm_gb_cgs_pass2", j, n, nnz) == ((k + 2) * V, 4 * k * n)
        assert bench.kernel_cost("gm_gc_cgs_pass3_givens", j, n, nnz) == ((k + 2) * V, 2 * k * n + 2 * n)
    # s = r - alpha v: two vectors in, one out, one FMA per row
    assert bench.kernel_cost("bcg_k2a_s_update", None, n, nnz) == (3 * V, 2 * n)


def test_recorded_traffic_follows_the_source_hash(monkeypatch):
    got = bench.recorded_traffic("gm_gb_cgs_pass2")
    if got is None:
        pytest.skip("profiles/dram_traffic.txt was taken on other kernel sources")
    assert 2.5e8 < got < 3.5e8  # one pass over 16-17 basis columns of 2.1 M rows
    monkeypatch.setattr(bench, "source_hash", lambda files=None: "0" * 16)
    assert bench.recorded_traffic("gm_gb_cgs_pass2") is None


def test_source_hash_covers_the_measured_kernels():
    import os

    d = os.path.join(bench.ROOT, "paper_0812_2769_gb300", "csrc")
    for fn in bench.TRAFFIC_SOURCES:
        assert os.path.exists(os.path.join(d, fn)), fn
    for fn in ("gmres_kernels.cuh", "bicgstab_kernels.cuh", "spmv_tma.cuh", "device_common.cuh"):
        assert fn in bench.TRAFFIC_SOURCES
    for fn in bench.GS_SOURCES:
        assert os.path.exists(os.path.join(d, fn)), fn
    assert "gs_spmv.cu" in bench.GS_SOURCES and "device_common.cuh" in bench.GS_SOURCES


def test_cpu_baseline_on_one_core_and_on_every_core():
    # the oracle in spawned single-threaded processes, on a small grid: one
    # process alone, then one per core of the affinity mask at once
    import os

    out = bench.cpu_sample(10, bcg_iters=2, gm_cycles=1, all_bcg_iters=2, all_gm_cycles=1)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert out["cores"] == min(len(os.sched_getaffinity(0)), bench.CpuOracle.MAX_PROCS)
    assert out["value"] > 0 and out["one_core"]["value"] > 0 and out["one_core"]["cores"] == 1
    # independent processes: all cores together beat one alone
    if out["cores"] > 1:
        assert out["value"] > out["one_core"]["value"]
