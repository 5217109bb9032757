#!/usr/bin/env python
"""Throughput benchmark of the GS(p) + Krylov hot path on one GB300.

Workload (one "step"): the 128^3 convection-diffusion system (2,097,152
unknowns, 14,581,760 nonzeros, 4x4x4 checkerboard a = 1 / 1e4, beta =
(20, 20, 20), seeded x_true, b = A x_true), freshly copied from a pristine
device copy, scaled by GS(2) and solved to a relative residual of 1e-8 (the
GS(2)-scaled metric of Sec. 2.2) twice: with Bi-CGSTAB and with GMRES(30).
Metric: solves per second (two solves per step).  The two solves of a step
are independent (both read the scaled A and b): they run concurrently on two
CUDA streams, each with its own library context, so that one solver's kernels
fill the SMs the other's leave idle at kernel boundaries.  The same steps
with the solves one after the other are timed as well ("serial" in the
line); --serial-solves runs only that form (the one to use under a
profiler, which serialises the two host threads' launches).

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) execute one
independent replica per GPU (weak scaling, no data-path collective); the
barrier and the max over ranks only frame the timing.

``--impl reference`` times the CPU oracle on a bounded sample of the same
workload instead (see cpu_sample()).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/sec and SpMV+Krylov HBM GB/s vs peak at rel. residual 1e-8; p50/p99 latency"
UNIT = "solves/s"
N_GRID = 128
TOL = 1e-8
M_GMRES = 30
FP64_PEAK_TFLOPS = 1.25  # nominal FP64 rate of GB300 (measured 1.19 TFLOP/s with an FMA probe)
SOLVES_PER_STEP = 2


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsk", choices=["gsk", "reference"])
    ap.add_argument("--grid", type=int, default=N_GRID, help="grid side (128 = the benchmark workload)")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel profiling pass")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the mixed-precision, batched (4096 systems) and serving measurements")
    ap.add_argument("--batch", type=int, default=4096, help="systems in the batched measurement")
    ap.add_argument("--serve-requests", type=int, default=120, help="requests in the serving measurement")
    ap.add_argument("--profile-kernels", choices=["gmres", "bicgstab", "both", "gs"], default=None,
                    help="only drive the solvers' kernels (or GS(p) alone) on the workload (for ncu captures)")
    ap.add_argument("--gs-calls", type=int, default=3, help="GS(p) calls per p in --profile-kernels gs")
    ap.add_argument("--gs-p", type=float, nargs="+", default=[2.0], help="the p of --profile-kernels gs")
    ap.add_argument("--gmres-iters", type=int, default=30, help="Arnoldi steps in --profile-kernels")
    ap.add_argument("--bicgstab-iters", type=int, default=20, help="Bi-CGSTAB iterations in --profile-kernels")
    ap.add_argument("--serial-solves", action="store_true",
                    help="run a step's two solves one after the other, and no concurrent step at all "
                         "(default: concurrently on two streams, the serial form timed beside it)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------- ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    """Largest value over all ranks (the slowest replica sets the job time)."""
    if dist is None:
        return value
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import tempfile

        self.gpu = gpu_index
        self.proc = None
        # raw samples: GSK_CLOCKS_DIR if set (to keep them), else a temp dir
        d = os.environ.get("GSK_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ---------------------------------------------------------------- workload
def workload(grid):
    from problems import configs

    return configs.c2(grid)


def config_dict(s, world):
    return {"workload": f"3D convection-diffusion {s.meta['N']}^3 (n={s.n}, nnz={s.nnz}), checkerboard 4^3 "
                        "a=1/1e4, beta=(20,20,20); GS(2) then Bi-CGSTAB and GMRES(30) to rel. residual 1e-8 "
                        "(GS(2)-scaled metric), FP64",
            "n": s.n, "nnz": s.nnz, "solves_per_step": SOLVES_PER_STEP, "parallelism": f"replicas x{world}",
            "solve_streams": 2,
            "l2": "inputs larger than L2 (A 183 MB + 8 working vectors of 16.8 MB)"}


def kernel_cost(name, step, n, nnz):
    """Algorithmic (bytes, FP64 flops) of one launch: every operand moved
    once (CSR int32 indices; x read once per product), no reuse counted."""
    spmv_b = 12 * nnz + 4 * (n + 1)
    V = 8 * n
    k = step + 1 if step is not None and step >= 0 else 1
    table = {
        "bcg_init": (spmv_b + 2 * V + 3 * V, 2 * nnz + 4 * n),
        "bcg_k1_spmv_dot": (spmv_b + 3 * V, 2 * nnz + 4 * n),
        "bcg_k2a_s_update": (3 * V, 2 * n),
        "bcg_k2b_spmv_dot": (spmv_b + 2 * V, 2 * nnz + 6 * n),
        "bcg_k3_xr_update": (7 * V, 10 * n),
        "bcg_k4_p_update": (4 * V, 4 * n),
        "bcg_kt_true_residual": (spmv_b + 3 * V, 2 * nnz + 4 * n),
        "bcg_kr_finish": (4 * V, 0),
        "gm_init_residual": (spmv_b + 3 * V, 2 * nnz + 4 * n),
        "gm_gr_restart_residual": (spmv_b + 3 * V, 2 * nnz + 4 * n),
        "gm_ga_spmv": (spmv_b + 2 * V, 2 * nnz + n),
        "gm_gd_cgs_pass1": ((k + 1) * V, 2 * k * n),
        "gm_gb_cgs_pass2": ((k + 2) * V, 4 * k * n),
        "gm_gc_cgs_pass3_givens": ((k + 2) * V, 2 * k * n + 2 * n),
        "gm_gx_x_update": ((k + 2) * V, 2 * k * n),
        "gm_gy_backsolve": (8 * (k * (k + 1) // 2 + 2 * k), k * k),
        "gs_norm(w)": (8 * nnz + 4 * (n + 1) + V, 2 * nnz),
        "unit_check": (V, 0),
    }
    return table.get(name, (0, 0))


# The sources that make the kernels of the traffic table and their launch
# shapes: the two solvers' translation units, everything they include, and
# the context (grid sizing); for GS(p), its translation unit.  Any edit to
# one of them voids the recorded traffic of those kernels (the ABI header,
# declarations only, does not enter).
TRAFFIC_SOURCES = ("gmres.cu", "bicgstab.cu", "ctx.cu", "gmres_kernels.cuh", "bicgstab_kernels.cuh", "spmv_tma.cuh",
                   "device_common.cuh", "internal.hpp", "graph.hpp", "ilu.cuh")
GS_SOURCES = ("gs_spmv.cu", "ctx.cu", "device_common.cuh", "internal.hpp")


def source_hash(files=TRAFFIC_SOURCES):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0812_2769_gb300", "csrc")
    for fn in files:
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, files=TRAFFIC_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash(files)
    for ln in open(path):
        p = ln.split()
        if len(p) >= 3 and not ln.startswith("#") and p[0] == kernel and p[2] == want:
            return float(p[1])
    return None


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    import paper_0812_2769_gb300 as g

    g.lib()
    dev = torch.device("cuda", local)
    s = workload(args.grid)
    val0 = torch.as_tensor(s.val, device=dev)
    b0 = torch.as_tensor(s.b, device=dev)
    A = g.Csr.from_host(s.rowptr, s.colidx, s.val, device=dev)
    b = b0.clone()
    x1 = torch.zeros(s.n, dtype=torch.float64, device=dev)
    x2 = torch.zeros_like(x1)
    ctx = g.Context(local)
    stream = torch.cuda.current_stream(dev)
    # the two solves of a step: own context (workspace, graphs) and stream each
    ctx_b, ctx_g = g.Context(local), g.Context(local)
    st_b, st_g = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    from concurrent.futures import ThreadPoolExecutor

    pool = ThreadPoolExecutor(max_workers=2)

    def solve_b(ev):
        # the library's calls release the interpreter lock while they wait
        st_b.wait_event(ev)
        with torch.cuda.stream(st_b):
            x1.zero_()
            return g.bicgstab_solve(A, b, x1, tol=TOL, ctx=ctx_b, stream=st_b)

    def solve_g(ev):
        st_g.wait_event(ev)
        with torch.cuda.stream(st_g):
            x2.zero_()
            return g.gmres_solve(A, b, x2, m=M_GMRES, tol=TOL, ctx=ctx_g, stream=st_g)

    def solves(serial):
        if serial:
            x1.zero_()
            i1 = g.bicgstab_solve(A, b, x1, tol=TOL, ctx=ctx)
            x2.zero_()
            i2 = g.gmres_solve(A, b, x2, m=M_GMRES, tol=TOL, ctx=ctx)
            return i1, i2
        ev = torch.cuda.Event()
        ev.record(stream)
        f1, f2 = pool.submit(solve_b, ev), pool.submit(solve_g, ev)
        i1, i2 = f1.result(), f2.result()
        stream.wait_stream(st_b)  # the next step overwrites A and b
        stream.wait_stream(st_g)
        return i1, i2

    def step(serial=args.serial_solves):
        A.val.copy_(val0)
        b.copy_(b0)
        g.gs_scale(A, b, p=2.0, ctx=ctx)
        return solves(serial)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    infos = []
    barrier(dist, local)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(dist, local)
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(dist, ms / 1e3)
    solves_done = sum_over_ranks(dist, SOLVES_PER_STEP * args.steps)
    value = solves_done / t_max

    # with the concurrent headline, the same steps with the solves one after
    # the other, same timing; their per-solve times are the solvers' own.
    # (--serial-solves runs no concurrent step at all: the form to use under
    # a profiler, which serialises the two host threads' launches.)
    other_line = None
    serial_infos = infos
    if not args.serial_solves:
        for _ in range(2):
            step(True)
        torch.cuda.synchronize()
        barrier(dist, local)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        serial_infos = [step(True) for _ in range(args.steps)]
        e3.record(stream)
        torch.cuda.synchronize()
        t_other = max_over_ranks(dist, e2.elapsed_time(e3) / 1e3)
        other_line = {"value": sum_over_ranks(dist, SOLVES_PER_STEP * args.steps) / t_other, "unit": UNIT,
                      "ms_per_step": t_other * 1e3 / args.steps}

    # kernels launched in the timed region, from each solve's counters and
    # the launch structure of its graph (kernels that return at entry count):
    # GS(2) one kernel; Bi-CGSTAB: weights, unit check and init, then a WHILE
    # body of 4 iterations x 5 kernels + kt + kr per pass, ceil(iters / 4)
    # passes between confirmations and one more per refresh; GMRES(30):
    # weights, unit check and init, then per cycle the 30 unrolled steps (4
    # kernels each: the product and the three CGS passes) and gy, gx, gr
    per_step = 4
    launches = 0
    for i1, i2 in infos:
        launches += 1
        launches += 3 + 22 * (math.ceil(i1["iters"] / 4) + i1["refreshes"])
        launches += 3 + (i2["restarts"] + 1) * (M_GMRES * per_step + 3)
    ok = all(i1["conv"] == g.CONVERGED and i2["conv"] == g.CONVERGED and i1["relres_true"] < TOL
             and i2["relres_true"] < TOL for i1, i2 in infos)

    # end to end through the public API from pinned host buffers
    e2e = None
    if True:  # every rank takes part (the max over ranks is a collective)
        rp_h = torch.as_tensor(s.rowptr).pin_memory()
        ci_h = torch.as_tensor(s.colidx).pin_memory()
        va_h = torch.as_tensor(s.val).pin_memory()
        b_h = torch.as_tensor(s.b).pin_memory()
        xo1 = torch.empty(s.n, dtype=torch.float64).pin_memory()
        xo2 = torch.empty_like(xo1)
        K = max(1, min(args.steps, 3))
        h2d = rp_h.numel() * 4 + ci_h.numel() * 4 + va_h.numel() * 8 + b_h.numel() * 8
        d2h = 2 * 8 * s.n

        def e2e_step():
            A.rowptr.copy_(rp_h, non_blocking=True)
            A.colidx.copy_(ci_h, non_blocking=True)
            A.val.copy_(va_h, non_blocking=True)
            b.copy_(b_h, non_blocking=True)
            g.gs_scale(A, b, p=2.0, ctx=ctx)
            solves(args.serial_solves)
            xo1.copy_(x1, non_blocking=True)
            xo2.copy_(x2, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()

        e2e_step()
        barrier(dist, local)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(K):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        t_e = max_over_ranks(dist, f0.elapsed_time(f1) / 1e3)
        e2e = {"value": sum_over_ranks(dist, SOLVES_PER_STEP * K) / t_e, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": K}

    roofline, kernels = None, None
    if not args.no_profile and rank == 0:
        roofline, kernels = profile_pass(g, ctx, A, val0, b, b0, s)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_sample(args.grid)

    extra = None
    if not args.no_extra and rank == 0:
        extra = {"mixed_precision": mixed_pass(g, ctx, A, val0, b, b0, x1, x2, args)}
        extra["batched"] = batched_pass(g, args)
        extra["c3_256"] = c3_pass(g)
        extra["serving"] = serving_pass(args)
        extra["spectrum"] = spectrum_pass(g, ctx, A, val0, b, b0, s)
        extra["ilu0"] = ilu_pass(g, ctx, A, val0, b, b0, s)
        extra["c1_32"] = c1_pass(g)
        extra["c2_scalings"] = c2_scalings_pass(g, ctx, A, val0, b, b0)
        extra["gs_scale_128"] = gs_pass(g, ctx, A, val0, b, b0, s)

    if rank == 0:
        # per-solve times from the serial steps (alone on the GPU, so per
        # iteration they compare kernels); counts and residuals are the same
        # in both modes
        i1, i2 = serial_infos[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": config_dict(s, world), "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "roofline": roofline, "cpu_baseline": cpu,
            "solves": {"bicgstab": dict({k: i1[k] for k in ("iters", "conv_name", "relres_true", "ms")},
                                        us_per_iter=round(1e3 * i1["ms"] / max(i1["iters"], 1), 2)),
                       "gmres30": dict({k: i2[k] for k in ("iters", "restarts", "conv_name", "relres_true", "ms")},
                                       us_per_step=round(1e3 * i2["ms"] / max(i2["iters"], 1), 2)),
                       "all_converged_below_tol": ok,
                       # Bi-CGSTAB's count on this system moves with the rounding
                       # of any summation order (240-370 seen): compare per iteration
                       "note": "iteration counts are rounding-sensitive; us_per_iter/us_per_step compare kernels",
                       "timing": "ms, us_per_iter, us_per_step from the serial steps (each solve alone)"},
            "solve_modes": ({"headline": "serial"} if args.serial_solves else
                            {"headline": "concurrent (two streams)", "serial": other_line}),
            "kernels": kernels,
            # the CSR product alone on the 256^3 matrix, the configuration
            # where it is purely bandwidth-bound (from forms.c3_256.spmv)
            "roofline_spmv": ({"kernel": "spmv_kernel (TMA ring), 256^3, FP64", "bound": "hbm",
                               "achieved": extra["c3_256"]["spmv"]["f64"]["GBps"], "peak": _peaks().get("hbm_gbs"),
                               "unit": "GB/s", "frac": extra["c3_256"]["spmv"]["f64"]["frac_of_measured_hbm"],
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
                              if extra and "c3_256" in extra else None),
            # GS(2) alone on the benchmark system (from forms.gs_scale_128)
            "roofline_gs": ({"kernel": "gs_rows_kernel (one pass), 128^3, p = 2", "bound": "hbm",
                             "achieved": extra["gs_scale_128"]["p2"]["GBps"], "peak": _peaks().get("hbm_gbs"),
                             "unit": "GB/s", "frac": extra["gs_scale_128"]["p2"]["frac_of_measured_hbm"],
                             "avg_us": extra["gs_scale_128"]["p2"]["us"],
                             "traffic": recorded_traffic("gs_rows_p2", GS_SOURCES),
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
                            if extra and "gs_scale_128" in extra else None),
            "forms": extra,
        }
        print(json.dumps(line), flush=True)
    pool.shutdown(wait=True)
    if dist is not None:
        dist.destroy_process_group()


def ilu_pass(g, ctx, A, val0, b, b0, s):
    """ILU(0) right preconditioning (level-scheduled sweeps) on the
    GS(2)-scaled workload: factorisation, one application, and a
    preconditioned Bi-CGSTAB solve to the same tolerance; plus the paper's
    Problem 1 row (Table 1, Bi-CGSTAB + ILUT with GS, 1e-10)."""
    import time

    import torch

    from paper_0812_2769_gb300 import reproduce
    from problems import configs

    A.val.copy_(val0)
    b.copy_(b0)
    g.gs_scale(A, b, p=2.0, ctx=ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M = g.Ilu0(A, ctx=ctx)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    r = b.clone()
    for _ in range(3):
        M.apply(r)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        M.apply(r)
    e1.record()
    torch.cuda.synchronize()
    x = torch.zeros_like(b)
    info = g.bicgstab_solve(A, b, x, tol=TOL, options=g.opts(precond=M), ctx=ctx)
    M.close()
    conv, it, rr, ms = reproduce.solve_case(g, configs.p1(128), "bicgstab", True, 1e-10, ctx=ctx, precond=True)
    return {"factor_s": round(t_factor, 3), "apply_ms": round(e0.elapsed_time(e1) / 10, 3),
            "bicgstab": {k: info[k] for k in ("iters", "conv_name", "relres_true", "ms")},
            "p1_table1_bicgstab_ilu_gs2_1e-10": {"converged": conv, "iters": it, "paper_iters": 130,
                                                 "relres_true": rr, "ms": round(ms, 1)}}


def spectrum_pass(g, ctx, A, val0, b, b0, s, m=64):
    """Ritz values of 64 Arnoldi steps (gsk_arnoldi) on the GS(2)-scaled
    workload: the eigenvalue diagnostic at a size no dense solver takes."""
    import time

    import numpy as np
    import torch

    A.val.copy_(val0)
    b.copy_(b0)
    g.gs_scale(A, b, p=2.0, ctx=ctx)
    v0 = torch.as_tensor(np.random.default_rng(0).normal(size=s.n), device=A.val.device)
    g.arnoldi(A, v0, m, ctx=ctx)  # warm-up (records the graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H, k = g.arnoldi(A, v0, m, ctx=ctx)
    sec = time.perf_counter() - t0
    ritz = np.linalg.eigvals(H[:k, :k])
    return {"steps": k, "ms": 1e3 * sec, "us_per_step": 1e6 * sec / max(k, 1),
            "ritz_lambda_max": float(np.abs(ritz).max()), "ritz_lambda_min": float(np.abs(ritz).min()),
            "note": "one graph launch (the m steps recorded once)"}


def mixed_pass(g, ctx, A, val0, b, b0, x1, x2, args):
    """The same step with the mixed-precision solvers (FP32 inner solves in
    FP64 refinement; the FP64 metric still has to fall below 1e-8)."""
    import torch

    o = g.opts(precision=g.PREC_MIXED)

    def step():
        A.val.copy_(val0)
        b.copy_(b0)
        g.gs_scale(A, b, p=2.0, ctx=ctx)
        x1.zero_()
        i1 = g.bicgstab_solve(A, b, x1, tol=TOL, options=o, ctx=ctx)
        x2.zero_()
        i2 = g.gmres_solve(A, b, x2, m=M_GMRES, tol=TOL, options=o, ctx=ctx)
        return i1, i2

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.steps)
    e0.record()
    infos = [step() for _ in range(K)]
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    i1, i2 = infos[-1]
    return {"value": SOLVES_PER_STEP * K / t, "unit": UNIT, "ms_per_step": 1e3 * t / K, "dtype": "f32 inner, f64 refinement",
            "solves": "one after the other (compare with solve_modes.serial of the FP64 headline)",
            "bicgstab": {k: i1[k] for k in ("iters", "refinements", "conv_name", "relres_true", "ms")},
            "gmres30": {k: i2[k] for k in ("iters", "refinements", "conv_name", "relres_true", "ms")},
            "all_converged_below_tol": all(a["conv"] == 0 and a["relres_true"] < TOL and c["conv"] == 0
                                           and c["relres_true"] < TOL for a, c in infos)}


def c3_pass(g, steps=2000):
    """The 256^3 configuration (coefficients 10^U[-3,3] on an 8^3 partition,
    convection U[-30,30]^3): GS(2), then GMRES(30) for a fixed number of
    Arnoldi steps in FP64 and with FP32 inner solves in FP64 refinement;
    time per step and the GS(2)-scaled residual reached (restarted GMRES(30)
    stagnates near 1e-7 on this system, so both run the same step count)."""
    import torch

    from problems import configs

    s = configs.c3(256)
    out = {"n": s.n, "nnz": s.nnz, "steps": steps}
    A = g.Csr.from_host(s.rowptr, s.colidx, s.val)
    val0 = A.val.clone()
    b0 = torch.as_tensor(s.b, device="cuda")
    b = b0.clone()
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    for name, prec in (("f64", g.PREC_F64), ("mixed", g.PREC_MIXED)):
        A.val.copy_(val0)
        b.copy_(b0)
        g.gs_scale(A, b, p=2.0)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = g.gmres_solve(A, b, x, m=M_GMRES, tol=1e-10, options=g.opts(precision=prec, maxit=steps))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": ms, "us_per_step": 1e3 * ms / max(1, info["iters"]), "iters": info["iters"],
                     "refinements": info["refinements"], "relres_true": info["relres_true"],
                     "conv_name": info["conv_name"]}
    # the CSR product alone on this matrix (the clean HBM-bound case): FP64
    # and FP32 values, algorithmic bytes (w + 4) nnz + 4 (n + 1) + 2 w n
    hbm = _peaks().get("hbm_gbs", 6800.0)
    spmv = {}
    for name, A1 in (("f64", A), ("f32", g.Csr(A.rowptr, A.colidx, A.val.float()))):
        xv = torch.ones(s.n, dtype=A1.val.dtype, device="cuda")
        yv = torch.empty_like(xv)
        for _ in range(3):
            g.gsk_spmv(A1, xv, yv)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            g.gsk_spmv(A1, xv, yv)
        e1.record()
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / 10
        w = A1.val.element_size()
        byt = (w + 4) * s.nnz + 4 * (s.n + 1) + 2 * w * s.n
        spmv[name] = {"us": round(us, 1), "algorithmic_MB": round(byt / 1e6, 1), "GBps": round(byt / us / 1e3, 1),
                      "frac_of_measured_hbm": round(byt / us / 1e3 / hbm, 3)}
        del xv, yv
    out["spmv"] = spmv
    # the solvers' kernels on this matrix, from a host loop with CUDA events
    # around each launch (one GMRES(30) cycle, 10 Bi-CGSTAB iterations): at
    # 16.8 M rows the fixed per-launch time weighs 8x less than at 128^3
    A.val.copy_(val0)
    b.copy_(b0)
    g.gs_scale(A, b, p=2.0)
    out["kernels"] = kernel_table(g, A, b, s.n, s.nnz, hbm, (("gmres", 30), ("bicgstab", 10)))
    # what the oracle reaches on the same system (written by
    # tests/golden/make_c3_oracle_trace.py): GMRES(30)'s metric after its first
    # two cycles, and Bi-CGSTAB over a rounding ensemble (none converges to
    # 1e-10 within 3,000 iterations)
    tr = os.path.join(ROOT, "tests", "golden", "c3_oracle_trace.json")
    if os.path.exists(tr):
        d = json.load(open(tr))
        out["oracle"] = {"gmres30_metric_after_cycles": [c["mu"] for c in d["gmres30"]["cycles"]],
                         "bicgstab_members": len(d["bicgstab"]),
                         "bicgstab_outcomes": sorted({r["conv"] for r in d["bicgstab"]}),
                         "bicgstab_metric_range": [min(r["relres_true"] for r in d["bicgstab"]),
                                                   max(r["relres_true"] for r in d["bicgstab"])],
                         "bicgstab_maxit": max(r["iters"] for r in d["bicgstab"])}
    del A, val0, b0, b, x
    torch.cuda.empty_cache()
    return out


def kernel_table(g, A, b, n, nnz, hbm, runs):
    """Per-kernel averages of gsk_profile_solve launches: us per launch,
    algorithmic GB/s and FP64 TFLOP/s (kernel_cost), fractions of the HBM
    and FP64 peaks."""
    import torch

    agg = {}
    for solver, iters in runs:
        x = torch.zeros(n, dtype=torch.float64, device=A.val.device)
        recs, _ = g.profile_solve(A, b, x, solver=solver, m=M_GMRES, tol=TOL, max_iters=iters)
        for name, step, ms in recs:
            by, fl = kernel_cost(name, step, n, nnz)
            a = agg.setdefault(name, [0, 0.0, 0.0, 0.0])
            a[0] += 1
            a[1] += ms
            a[2] += by
            a[3] += fl
        del x
    out = {}
    for name, (k, ms, by, fl) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        t = ms / 1e3
        if t <= 0 or by <= 0:
            continue
        out[name] = {"launches": k, "us": round(1e6 * t / k, 1), "GBps": round(by / t / 1e9, 1),
                     "hbm_frac": round(by / t / 1e9 / hbm, 3), "fp64_frac": round(fl / t / 1e12 / FP64_PEAK_TFLOPS, 3)}
    return out


def _peaks():
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pk)) if os.path.exists(pk) else {}


def c1_pass(g):
    """The 32^2 configuration: latency-bound (the system fits in L2), so
    microseconds per solve rather than a bandwidth fraction: GMRES(20) and
    Bi-CGSTAB, unscaled and after GS(2), to 1e-8.  Both solvers run a system
    this small on one thread-block cluster; each is timed on the grid-wide
    path too (a context created with GSK_SMALL_N=0)."""
    import torch

    from problems import configs

    s = configs.c1()
    A = g.Csr.from_host(s.rowptr, s.colidx, s.val)
    val0 = A.val.clone()
    b0 = torch.as_tensor(s.b, device="cuda")
    b = b0.clone()
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    ctx = g.Context(torch.cuda.current_device())
    old = os.environ.get("GSK_SMALL_N")
    os.environ["GSK_SMALL_N"] = "0"
    try:
        ctx_grid = g.Context(torch.cuda.current_device())
    finally:
        if old is None:
            del os.environ["GSK_SMALL_N"]
        else:
            os.environ["GSK_SMALL_N"] = old
    out = {"n": s.n, "nnz": s.nnz, "cluster_path_rows": g.small_system_rows(ctx)}
    for scaled in (False, True):
        A.val.copy_(val0)
        b.copy_(b0)
        if scaled:
            g.gs_scale(A, b, p=2.0, ctx=ctx)
        for solver in ("gmres20", "gmres20_grid_wide", "bicgstab", "bicgstab_grid_wide"):
            c = ctx_grid if solver.endswith("wide") else ctx
            # GMRES(20) stagnates here (10,000 steps); the grid-wide run
            # stops at 2,000 to keep the bench short: compare us_per_iter
            o = g.opts(maxit=2000) if solver == "gmres20_grid_wide" else None

            def solve():
                x.zero_()
                if solver.startswith("gmres20"):
                    return g.gmres_solve(A, b, x, m=20, tol=TOL, options=o, ctx=c)
                return g.bicgstab_solve(A, b, x, tol=TOL, ctx=c)
            reps = 3 if solver.startswith("gmres20") else 20
            for _ in range(2):
                info = solve()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                info = solve()
            dt = (time.perf_counter() - t0) / reps
            out[("gs2_" if scaled else "unscaled_") + solver] = {
                "us_per_solve": round(1e6 * dt, 1), "solves_per_s": round(1 / dt, 1), "iters": info["iters"],
                "us_per_iter": round(1e6 * dt / max(info["iters"], 1), 2),
                "conv_name": info["conv_name"], "relres_true": info["relres_true"]}
    ctx_grid.close()
    return out


def c2_scalings_pass(g, ctx, A, val0, b, b0):
    """The benchmark system under the other scalings the configuration names:
    unscaled, GS(1) and GS(inf) (GS(2) is the headline); both solvers to 1e-8,
    at most 10,000 iterations."""
    import torch

    out = {}
    for name, p in (("unscaled", None), ("gs1", 1.0), ("gs_inf", math.inf)):
        row = {}
        for solver in ("bicgstab", "gmres30"):
            A.val.copy_(val0)
            b.copy_(b0)
            if p is not None:
                g.gs_scale(A, b, p=p, ctx=ctx)
            x = torch.zeros_like(b)
            info = (g.gmres_solve(A, b, x, m=M_GMRES, tol=TOL, ctx=ctx) if solver == "gmres30"
                    else g.bicgstab_solve(A, b, x, tol=TOL, ctx=ctx))
            row[solver] = {k: info[k] for k in ("iters", "conv_name", "relres_true", "ms")}
        out[name] = row
    return out


def batched_pass(g, args):
    """The batch configuration: args.batch 2D inclusion systems (side 16..128),
    GS(2) + Bi-CGSTAB to 1e-8 in one persistent launch, FP64 and mixed,
    against a loop of single-system FP64 solves on the first 128 systems."""
    import torch

    from problems import configs

    systems = [configs.c4_system(i) for i in range(args.batch)]
    val0 = [torch.as_tensor(x.val, device="cuda") for x in systems]
    b0 = [torch.as_tensor(x.b, device="cuda") for x in systems]
    As = [g.Csr.from_host(x.rowptr, x.colidx, x.val) for x in systems]
    bs = [v.clone() for v in b0]
    xs = [torch.zeros(x.n, dtype=torch.float64, device="cuda") for x in systems]
    from paper_0812_2769_gb300 import autotune

    ctx = g.Context(torch.cuda.current_device())
    out = {"systems": len(systems), "unknowns": int(sum(x.n for x in systems)),
           "nnz": int(sum(x.nnz for x in systems))}

    def reset(k=None):
        for A, v, bb, b1, x in list(zip(As, val0, b0, bs, xs))[:k]:
            A.val.copy_(v)
            b1.copy_(bb)
            x.zero_()
        torch.cuda.synchronize()

    def timed(prec, cfg, solver="bicgstab", k=None, maxit=10000):
        best, infos = None, None
        for _ in range(2):
            reset(k)
            o = g.opts(precision=prec, maxit=maxit, **cfg)
            if solver == "gmres":
                infos, _ = g.gmres_solve_batched(As[:k], bs[:k], xs[:k], m=M_GMRES, p=2.0, tol=TOL, options=o, ctx=ctx)
            else:
                infos, _ = g.bicgstab_solve_batched(As[:k], bs[:k], xs[:k], p=2.0, tol=TOL, options=o, ctx=ctx)
            ms = infos[0]["ms"]
            best = ms if best is None else min(best, ms)
        return best, infos

    for name, prec in (("f64", g.PREC_F64), ("mixed", g.PREC_MIXED)):
        reset()
        t0 = time.perf_counter()
        cfg = autotune.batched_config(As, bs, xs, solver="bicgstab", p=2.0, tol=TOL, precision=prec, reps=1)
        t_tune = time.perf_counter() - t0
        cfg = {k: cfg[k] for k in ("batch_block", "batch_large_n")}
        best, infos = timed(prec, cfg)
        default_ms, _ = timed(prec, {})
        out[name] = {"value": len(systems) / (best / 1e3), "unit": UNIT, "ms": best,
                     "converged": sum(i["conv"] == g.CONVERGED for i in infos),
                     "iters_mean": float(sum(i["iters"] for i in infos) / len(infos)),
                     "autotuned": cfg, "tuning_seconds": round(t_tune, 2), "default_shape_ms": default_ms}
    # per-iteration cost of the two arithmetic forms, from two fixed
    # iteration counts (tol 0: a system runs to maxit unless it breaks down):
    # FP64 Bi-CGSTAB iterations, and the FP32 iterations of the mixed form
    # (one inner solve of maxit iterations, inner_tol 1e-300); the slope
    # between the two counts leaves out GS, the FP32 copy of the matrix and
    # the residuals
    per = {}
    for name, prec in (("f64", g.PREC_F64), ("f32_inner", g.PREC_MIXED)):
        pts = []
        for M in (20, 60):
            reset()
            o = g.opts(precision=prec, maxit=M, inner_maxit=M, inner_tol=1e-300)
            infos, _ = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=0.0, options=o, ctx=ctx)
            pts.append((sum(i["iters"] for i in infos), infos[0]["ms"]))
        (i1, t1), (i2, t2) = pts
        per[name] = {"ns_per_system_iteration": round(1e6 * (t2 - t1) / max(i2 - i1, 1), 3),
                     "system_iterations": [i1, i2], "ms": [round(t1, 3), round(t2, 3)]}
    per["f32_over_f64"] = round(per["f32_inner"]["ns_per_system_iteration"] / per["f64"]["ns_per_system_iteration"], 3)
    out["per_iteration"] = per
    # batched GMRES(30), FP64, on the first 1024 systems (restarted GMRES
    # stagnates on many of these inclusion systems: capped at 1000 steps)
    K = min(1024, len(systems))
    gm_ms, gm_infos = timed(g.PREC_F64, {}, solver="gmres", k=K, maxit=1000)
    out["gmres30_f64"] = {"systems": K, "maxit": 1000, "ms": gm_ms, "value": K / (gm_ms / 1e3), "unit": UNIT,
                          "converged": sum(i["conv"] == g.CONVERGED for i in gm_infos),
                          "iters_mean": float(sum(i["iters"] for i in gm_infos) / len(gm_infos))}
    K = min(128, len(systems))
    for A, v, bb, b1, x in zip(As[:K], val0[:K], b0[:K], bs[:K], xs[:K]):
        A.val.copy_(v)
        b1.copy_(bb)
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for A, b1, x in zip(As[:K], bs[:K], xs[:K]):
        g.gs_scale(A, b1, p=2.0, ctx=ctx)
        g.bicgstab_solve(A, b1, x, tol=TOL, ctx=ctx)
    torch.cuda.synchronize()
    out["per_system_loop_f64"] = {"value": K / (time.perf_counter() - t0), "unit": UNIT, "systems": K}
    return out


def serving_pass(args):
    """Serving: mixed 2D/3D requests (see problems/serving.py), mixed
    precision to 1e-8.  The capacity is measured with every request queued at
    once; then the same requests arrive as a Poisson stream at 50%, 80% and
    95% of it, each run reporting p50/p99 latency (arrival to completion) over
    the converged solves, with the sample count.  Beside it, the same queued
    requests through the same server in FP64, and through a plain loop of FP64
    calls (upload, GS, solve, read back x; one context, one stream)."""
    import torch

    import paper_0812_2769_gb300 as g
    from paper_0812_2769_gb300 import serve
    from problems import serving as sv

    n = args.serve_requests
    specs = sv.stream(n, rate=1.0, seed=7)
    systems = [sp.build() for sp in specs]

    def requests(rate, precision="mixed"):
        # the stream's request mix does not depend on its rate, only the arrival times
        arr = [sp.arrival for sp in sv.stream(n, rate=rate, seed=7)] if rate else [0.0] * n
        return [serve.Request(sp.rid, sysm, solver=sp.solver, m=sp.m, p=sp.p, tol=TOL, precision=precision,
                              arrival=t, maxit=3000) for sp, sysm, t in zip(specs, systems, arr)]

    be = serve.GpuBackend(0, slots=6)
    serve.Server(be, slots=6).run(requests(None)[:3], realtime=False)  # warm the contexts
    sat = serve.summarize(serve.Server(be, slots=6).run(requests(None), realtime=False))
    capacity = sat["solves_per_s"]
    sat64 = serve.summarize(serve.Server(be, slots=6).run(requests(None, "f64"), realtime=False))
    loads = {}
    for f in (0.5, 0.8, 0.95):
        srv = serve.Server(be, slots=6)
        out = serve.summarize(srv.run(requests(f * capacity), realtime=True))
        out.update({"arrival_rate_per_s": round(f * capacity, 3), "peak_admitted_GB": round(srv.peak_in_use / 1e9, 3)})
        loads[f"{round(100 * f)}%"] = out

    # the plain FP64 loop: what a caller without the server does per request
    ctx = g.Context(0)
    o = g.opts(precision=g.PREC_F64, maxit=3000)
    conv = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sp, sysm in zip(specs, systems):
        A = g.Csr.from_host(sysm.rowptr, sysm.colidx, sysm.val)
        b = torch.as_tensor(sysm.b, device="cuda")
        x = torch.zeros(sysm.n, dtype=torch.float64, device="cuda")
        g.gs_scale(A, b, p=sp.p, ctx=ctx)
        if sp.solver == "gmres":
            info = g.gmres_solve(A, b, x, m=sp.m, tol=TOL, options=o, ctx=ctx)
        else:
            info = g.bicgstab_solve(A, b, x, tol=TOL, options=o, ctx=ctx)
        x.cpu()
        conv += info["conv"] == g.CONVERGED
    t_loop = time.perf_counter() - t0
    ctx.close()
    keys = ("completed", "converged", "solves_per_s", "p50_s", "p99_s", "latency_samples", "lanes")
    return {"requests_per_run": n, "slots": 6, "maxit": 3000, "capacity_solves_per_s": capacity,
            "capacity_run": {k: sat[k] for k in keys},
            "fp64_server": {k: sat64[k] for k in keys},
            "fp64_loop": {"converged": int(conv), "solves_per_s": conv / t_loop, "seconds": round(t_loop, 3),
                          "note": "one request after another: upload, GS, FP64 solve, read back x"},
            "loads": loads}


def gs_pass(g, ctx, A, val0, b, b0, s, reps=10):
    """GS(p) alone on the benchmark system, p = 2, 1 and inf: the device time
    of the fused one-pass kernel from CUDA events around its launch on the
    bench stream (gsk_profile_gs_scale; A and b restored before each call,
    which also pushes most of the 275 MB the kernel moves out of L2), and the
    whole gs_scale call (clearing the error word, the kernel, the read-back
    that synchronises) timed by events around it.  Algorithmic bytes per
    call: rowptr, the values and b read once, the values and b written once."""
    import torch

    hbm = float(_peaks().get("hbm_gbs", 6800.0))
    st = torch.cuda.current_stream()
    by = 4 * (s.n + 1) + 16 * s.nnz + 16 * s.n
    out = {"algorithmic_bytes": by}
    for name, p in (("p2", 2.0), ("p1", 1.0), ("p_inf", math.inf)):
        kern, call = [], []
        for i in range(3 + reps):
            A.val.copy_(val0)
            b.copy_(b0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ms = g.profile_gs_scale(A, b, p=p, ctx=ctx, stream=st)
            e1.record(st)
            e1.synchronize()
            if i >= 3:
                kern.append(ms / 1e3)
                call.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.mean(kern)
        out[name] = {"us": round(1e6 * t, 2), "GBps": round(by / t / 1e9, 1),
                     "frac_of_measured_hbm": round(by / t / 1e9 / hbm, 4),
                     "call_us": round(1e6 * statistics.mean(call), 2)}
    return out


def profile_pass(g, ctx, A, val0, b, b0, s):
    """Per-kernel device times from CUDA events around each launch (the same
    kernels driven from a host loop), for the roofline of the dominant one."""
    import torch

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    A.val.copy_(val0)
    b.copy_(b0)
    g.gs_scale(A, b, p=2.0, ctx=ctx)
    agg = {}
    for solver in ("bicgstab", "gmres"):
        x = torch.zeros(s.n, dtype=torch.float64, device=A.val.device)
        recs, info = g.profile_solve(A, b, x, solver=solver, m=M_GMRES, tol=TOL, max_iters=10000, ctx=ctx)
        for name, step, ms in recs:
            by, fl = kernel_cost(name, step, s.n, s.nnz)
            a = agg.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            a["launches"] += 1
            a["ms"] += ms
            a["bytes"] += by
            a["flops"] += fl
    total = sum(a["ms"] for a in agg.values())
    kernels = {}
    for name, a in sorted(agg.items(), key=lambda kv: -kv[1]["ms"]):
        t = a["ms"] / 1e3
        kernels[name] = {"launches": a["launches"], "ms_total": round(a["ms"], 3),
                         "share": round(a["ms"] / total, 4),
                         "GBps": round(a["bytes"] / t / 1e9, 1) if t > 0 else None,
                         "fp64_TFLOPs": round(a["flops"] / t / 1e12, 4) if t > 0 else None}
    dom, a = max(agg.items(), key=lambda kv: kv[1]["ms"])
    t_avg = a["ms"] / a["launches"] / 1e3
    gbs = a["bytes"] / a["launches"] / t_avg / 1e9
    tfl = a["flops"] / a["launches"] / t_avg / 1e12
    f_hbm, f_alu = gbs / hbm, tfl / FP64_PEAK_TFLOPS
    if f_alu > f_hbm:
        roof = {"bound": "alu", "achieved": round(tfl, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(f_alu, 4), "peak_source": "nominal GB300 FP64 rate (FMA probe measured 1.19)"}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(f_hbm, 4),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof.update({"kernel": dom, "launches": a["launches"], "avg_us": round(t_avg * 1e6, 2),
                 "share": kernels[dom]["share"], "hbm_frac": round(f_hbm, 4), "fp64_frac": round(f_alu, 4),
                 "traffic": recorded_traffic(dom),
                 "timing": "CUDA events around each launch, kernels driven from a host loop on the bench stream"})
    return roof, kernels


# ---------------------------------------------------------------- CPU oracle
_CPU_SYS = {}


def _cpu_init(grid):
    """Worker set-up: the workload and its GS(2) scaling, once per process."""
    import oracle

    s = workload(grid)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    _CPU_SYS["s"], _CPU_SYS["val"], _CPU_SYS["b"] = s, val, b


def _cpu_task(args):
    """One bounded oracle sample (one thread): per-iteration and per-cycle
    seconds of Bi-CGSTAB and GMRES(30), and GS(2) seconds."""
    import oracle

    bcg_iters, gm_cycles = args
    s, val, b = _CPU_SYS["s"], _CPU_SYS["val"], _CPU_SYS["b"]
    t0 = time.perf_counter()
    oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    t_gs = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=TOL, maxit=bcg_iters)
    t_b = (time.perf_counter() - t0) / bcg_iters
    t0 = time.perf_counter()
    oracle.gmres(s.rowptr, s.colidx, val, b, m=M_GMRES, tol=TOL, maxit=M_GMRES * gm_cycles)
    t_cyc = (time.perf_counter() - t0) / gm_cycles
    return t_gs, t_b, t_cyc


def _cpu_step_seconds(t_gs, t_b, t_cyc):
    """Seconds of one step (GS(2) + both solves) from a sample, scaled by the
    oracle's own iteration counts for this workload."""
    counts = json.load(open(os.path.join(ROOT, "tests", "golden", "c2_oracle_counts.json")))
    nb, ng = counts["bicgstab"]["iters"], counts["gmres30"]["iters"]
    return t_gs + t_b * nb + t_cyc * math.ceil(ng / M_GMRES), nb, ng


class CpuOracle:
    """The plain single-threaded oracle on the host: one process alone (one
    core), and one process per core of the affinity mask at once (the host's
    throughput: independent solves, the oracle itself unthreaded; at most
    MAX_PROCS processes, about 1 GB each at 128^3).  Processes are spawned
    (never forked after CUDA has started); every wait on them is bounded."""

    MAX_PROCS = 32
    TIMEOUT_S = 600

    def __init__(self, grid):
        import multiprocessing as mp

        self.cores = min(len(os.sched_getaffinity(0)), self.MAX_PROCS)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_cpu_init, initargs=(grid,))
        # every worker builds its workload before the first timed sample
        self.pool.map_async(_cpu_task, [(1, 1)] * self.cores, chunksize=1).get(self.TIMEOUT_S)

    def one_core(self, bcg_iters, gm_cycles):
        return self.pool.apply_async(_cpu_task, ((bcg_iters, gm_cycles),)).get(self.TIMEOUT_S)

    def all_cores(self, bcg_iters, gm_cycles):
        return self.pool.map_async(_cpu_task, [(bcg_iters, gm_cycles)] * self.cores,
                                   chunksize=1).get(self.TIMEOUT_S)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_sample(grid, bcg_iters=80, gm_cycles=3, all_bcg_iters=40, all_gm_cycles=1):
    """The CPU oracle on a bounded sample of the workload: GS(2), bcg_iters
    Bi-CGSTAB iterations and gm_cycles full GMRES(30) cycles on one core
    (about 20 s), scaled to whole solves by the oracle's own iteration counts
    (tests/golden/c2_oracle_counts.json); then a shorter sample on every core
    of the affinity mask at once (one independent sample per core), which is
    the reported value."""
    import platform

    cpu = CpuOracle(grid)
    try:
        t1, nb, ng = _cpu_step_seconds(*cpu.one_core(bcg_iters, gm_cycles))
        t_all = [_cpu_step_seconds(*r)[0] for r in cpu.all_cores(all_bcg_iters, all_gm_cycles)]
    finally:
        cpu.close()
    all_rate = sum(SOLVES_PER_STEP / t for t in t_all)
    model = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    # Arm reports a part number: name the ones of this family
    model = {"0xd4f": "Arm Neoverse V2 (cpu part 0xd4f)", "0xd8e": "Arm Neoverse V3 (cpu part 0xd8e)"}.get(model, model)
    return {"value": all_rate, "unit": UNIT, "cores": cpu.cores, "kind": "oracle", "cpu": model,
            "sample": f"GS(2) + {all_bcg_iters} Bi-CGSTAB iterations + {all_gm_cycles} GMRES(30) cycle(s) on "
                      f"the 128^3 workload in each of {cpu.cores} single-threaded oracle processes at once, "
                      f"scaled to {nb} Bi-CGSTAB iterations and {ng} GMRES steps (the oracle's own counts)",
            "one_core": {"value": SOLVES_PER_STEP / t1, "unit": UNIT, "cores": 1,
                         "sample": f"GS(2) + {bcg_iters} Bi-CGSTAB iterations + {gm_cycles} GMRES(30) cycles, "
                                   f"one process alone"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s = workload(args.grid)
    cpu = CpuOracle(args.grid)
    samples = []
    try:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = cpu.all_cores(10, 1)
            if i >= args.warmup:
                rate = sum(SOLVES_PER_STEP / _cpu_step_seconds(*r)[0] for r in res)
                samples.append((rate, time.perf_counter() - t0))
    finally:
        cpu.close()
    val = statistics.mean(r for r, _ in samples)
    sample = (f"per step: GS(2) + 10 Bi-CGSTAB iterations + 1 GMRES(30) cycle on the 128^3 workload in each of "
              f"{cpu.cores} single-threaded oracle processes at once, scaled to whole solves by the oracle's "
              f"own iteration counts")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(t for _, t in samples), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": config_dict(s, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_kernels(args):
    """Kernel-only run for ncu: GS(2) on the workload, then the FP64 solvers'
    kernels driven from a host loop for a fixed number of iterations; with
    "gs", GS(p) alone --gs-calls times on the pristine workload, for each p of
    --gs-p (the matrix restored between calls)."""
    import torch

    import paper_0812_2769_gb300 as g

    s = workload(args.grid)
    A = g.Csr.from_host(s.rowptr, s.colidx, s.val)
    b = torch.as_tensor(s.b, device="cuda")
    if args.profile_kernels == "gs":
        val0, b0 = A.val.clone(), b.clone()
        for p in args.gs_p:
            for _ in range(args.gs_calls):
                A.val.copy_(val0)
                b.copy_(b0)
                ms = g.profile_gs_scale(A, b, p=p)
                print(f"gs p={p:g} kernel {1e3 * ms:.1f} us")
        return
    g.gs_scale(A, b, p=2.0)
    for solver, iters in (("gmres", args.gmres_iters), ("bicgstab", args.bicgstab_iters)):
        if args.profile_kernels in (solver, "both"):
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            recs, info = g.profile_solve(A, b, x, solver=solver, m=M_GMRES, tol=TOL, max_iters=iters)
            print(solver, len(recs), "launches", info["iters"], "iterations")


def main(argv=None):
    args = parse_args(argv)
    if args.profile_kernels:
        profile_kernels(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
