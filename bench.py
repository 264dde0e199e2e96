"""Benchmark of the GB300 cut-cell multigrid solve (one JSON line on rank 0).

Workload: the unit square minus the disk of radius 0.2 at (0.5, 0.5),
a u_xx + b u_xy + c u_yy = f with (a, b, c) = (1, 0.5, 2), Dirichlet data on
the box and Neumann data on the circle, manufactured u = exp(x) cos(2y), on
1024 x 1024 cells (the finest grid of the disk refinement sweep).  A step is
one whole solve through the C ABI: assembly of b = f - N g, then FP32 W(4,4)
cycles (gamma = 2 on the finest level only) inside FP64 iterative
refinement until ||b - A u||_inf / ||b||_inf < 1e-13, from u = 0.  That tolerance is what discretisation-error accuracy takes
on this workload: ||b||_inf grows like h^-2 (boundary data enters b through
the ghost formulas), and at 1e-10 the algebraic error (4e-9 max-norm) is far
above the discretisation error at every N from 256 up, while at 1e-13 the
error reaches the FP64 round-off floor (1.5e-11 at 1024^2; 7e-12 at 512^2).
Setup (cut cells, fits, factorisations) runs once before timing, as it does
for a cached hierarchy.

Timing: CUDA events around every step on the solve stream; an L2 flush (a
512 MB write) runs between steps outside the events.  `value` is the solved
DOF/s of the whole job (all ranks).  `e2e` is the same metric through
cc_solve_host from pinned host memory, copies included.

--impl reference times the FP64 CPU oracle (the method as a plain numpy /
scipy program) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 1024
TOL = 1e-13
MIN_COARSE = 32
# W(4,4) with the W-cycle's repeated coarse-grid correction on the finest
# level only (gamma = 2 there, V below): at 1024^2 it needs 22 cycles and
# 4361 launches per solve, against 26 cycles and 6193 launches for W(3,3)
# repeated on the 2 finest levels and 11,975 for the full W(3,3)
NU = 4
W_DEPTH = 1
# the random-domain batch is also solved with the Krylov outer iteration
# (cc_options.krylov): FGMRES(20) preconditioned by the same cycle in FP64
# (an FP32 cycle keeps too few digits where the cycle alone diverges)
KRYLOV = 20
KRYLOV_MAX_CYCLES = 400
# DRAM bytes per timed interval (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture (cold caches), keyed like cc_kernel_timing's kernels:
# k_sweep_p per 1024^2 launch (profiles/k_sweep_p_poisson4096_disk1024.md);
# the finest-level block solve of the 1024^2 disk with its autotuned chunk
# size, k_block_p1 + k_block_p2 (profiles/block_solve_p1p2_disk1024.md); the
# all-level block solves were not captured as one unit
TRAFFIC = {1: 9.46e6, 2: None, 3: 2.727e6 + 1.758e6}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", type=int, default=120,
                    help="requests in the serving measurement (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="mean arrival rate of the serving measurement, requests per second")
    ap.add_argument("--random-domains", type=int, default=16,
                    help="problems of the batch-workload measurement (0: skip)")
    ap.add_argument("--ellipse-union", type=int, nargs="*", default=[2048, 4096],
                    help="grids of the ellipse-union measurement (none: skip)")
    ap.add_argument("--hbm-n", type=int, default=4096,
                    help="grid of the HBM-bound sweep measurement (0: skip)")
    ap.add_argument("--serve-full", type=int, default=0, metavar="N",
                    help="run the full serving workload with N requests per rate (10000 as specified; "
                         "0: skip, the default, as it takes about a quarter of an hour)")
    ap.add_argument("--serve-domains", type=int, default=64)
    ap.add_argument("--serve-full-fp64", type=int, default=3000,
                    help="requests per rate of the FP64 arm of --serve-full (it runs at about a sixth "
                         "of the mixed arm's rate)")
    ap.add_argument("--serve-full-rates", default="100,300,1000,3000,5000")
    ap.add_argument("--plain", type=int, default=1,
                    help="also run the plain-method cases: Poisson 64^2 (and 1024^2, 4096^2) V(3,3), "
                         "the disk refinement sweep 128^2..1024^2, the Table 8 rates (0: skip)")
    ap.add_argument("--setup", type=int, default=1,
                    help="also time the setup with its per-cell steps on the device and on host "
                         "threads (0: skip)")
    ap.add_argument("--mcgs", type=int, default=1,
                    help="also time the headline problem with the multicolour smoother (0: skip)")
    ap.add_argument("--batch", type=int, default=8,
                    help="independent solves in the concurrent-batch measurement (0: skip)")
    ap.add_argument("--min-coarse", type=int, default=MIN_COARSE,
                    help="cells a side of the coarsest level")
    ap.add_argument("--profile-sweep", type=int, default=0, metavar="N",
                    help="set up the Poisson unit-square hierarchy at N^2 and run one mixed cycle "
                         "without graphs, then exit (for ncu -k regex:k_sweep_p)")
    ap.add_argument("--profile", action="store_true",
                    help="warm up, then run one solve inside the NVTX range 'solve' and exit "
                         "(for ncu --nvtx --nvtx-include solve/)")
    return ap.parse_args()


def run_profile(a):
    import torch

    import __graft_entry__
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I
    __graft_entry__.build()
    P = _problem()
    n = a.n
    # the host loop: every iteration is an ordinary graph launch, whose kernel
    # nodes ncu profiles one by one (the kernels are those of the loop graph,
    # without its one-thread convergence kernels)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=a.min_coarse, cycle=2, precision=1,
                                              max_cycles=60, w_depth=W_DEPTH, nu1=NU, nu2=NU,
                                              device_loop=0))
    f, g, _ = I.problem_inputs(H, P)
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device="cuda")
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    for _ in range(max(1, a.warmup)):
        u.zero_()
        H.solve(ft, gt, u, TOL)
    torch.cuda.synchronize()
    u.zero_()
    torch.cuda.nvtx.range_push("solve")
    r = H.solve(ft, gt, u, TOL)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile": "one solve", "n": n, "status": r.status, "cycles": r.cycles,
                      "kernels": r.kernels, "rel_res": r.rel_res,
                      "sweep_ctas": [H.info.sweep_ctas[l] for l in range(H.info.n_levels)],
                      "block_chunk_rows": [H.info.block_chunk_rows[l] for l in range(H.info.n_levels)]}))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to $BENCH_CLOCKS_DIR (default _bench_out/); the JSON
        # line carries their summary
        out = os.environ.get("BENCH_CLOCKS_DIR", os.path.join(ROOT, "_bench_out"))
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    """Rank, world size and a max-over-ranks reducer (torchrun or single)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world == 1:
        return rank, world, local, (lambda x: x), (lambda: None)
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    dev = torch.device("cuda", local) if backend == "nccl" else torch.device("cpu")

    def red_max(x: float) -> float:
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return rank, world, local, red_max, dist.barrier


def aggregate(dof_per_rank: float, ms_per_step_max: float, world: int) -> float:
    """Whole-job DOF/s: every rank solves its own problem per step."""
    return dof_per_rank * world / (ms_per_step_max / 1e3)


def _problem():
    import workloads as W
    return W.problem_disk()


# ---------------------------------------------------------------------------
def run_ours(a):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I

    rank, world, local, red_max, barrier = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    barrier()
    __graft_entry__.build()
    P = _problem()
    n = a.n
    opts = default_options(min_coarse_n=a.min_coarse, cycle=2, precision=1, max_cycles=60,
                           w_depth=W_DEPTH, nu1=NU, nu2=NU)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, opts)
    f, g, ue = I.problem_inputs(H, P)
    present = H.cell_types()[0] != 0
    dof = int(H.info.n_dof)
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device=dev)
    gt = torch.tensor(g, dtype=torch.float64, device=dev)
    u = torch.zeros(n * n, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        u.zero_()
        r = H.solve(ft, gt, u, TOL, stream)
        if r.status != 0:
            raise RuntimeError(f"solve failed: status {r.status}, rel_res {r.rel_res}")
        return r

    for _ in range(a.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    err = float(np.abs(u.cpu().numpy().reshape(n, n) - ue)[present].max())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    cycles, kernels = [], 0
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(a.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            r = step()
            ev[k][1].record(stream)
            cycles.append(r.cycles)
            kernels += r.kernels
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    ms = red_max(sum(step_ms) / a.steps)
    value = aggregate(dof, ms, world)

    # end to end: pinned host buffers through cc_solve_host
    hf = torch.tensor(f.ravel(), dtype=torch.float64).pin_memory().numpy()
    hg = torch.tensor(g, dtype=torch.float64).pin_memory().numpy()
    hu = torch.zeros(n * n, dtype=torch.float64).pin_memory().numpy()
    for _ in range(max(1, a.warmup)):
        hu[:] = 0
        H.solve_host(hf, hg, hu, TOL, stream)
    e2e_ms = []
    for _ in range(a.steps):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        hu[:] = 0
        t = time.perf_counter()
        r = H.solve_host(hf, hg, hu, TOL, stream)
        e2e_ms.append((time.perf_counter() - t) * 1e3)
        assert r.status == 0
    e2e = aggregate(dof, red_max(sum(e2e_ms) / len(e2e_ms)), world)

    # rooflines, from CUDA events recorded inside the solve graph on its
    # stream around each timed launch (each interval includes the launch
    # latency): the exact block solves (every level, one interval per solve:
    # its one dense launch or its two chunked launches) and the finest-level
    # FP32 Jacobi sweep; the one with more time per solve is the dominant
    # kernel.  `achieved` divides the method's algorithmic bytes (the block
    # solve priced as the paper's banded factors plus the gather, the sweep
    # as 3 x 4 B per cell) by the event time; `moved_gbs` divides the bytes
    # the library's kernels move.
    peaks, src = _peaks()
    peak = float(peaks["hbm_gbs"])
    roofs = {}
    for which, name in ((3, "exact block solve of the finest level (a2 + a3): k_block_p1<float> + "
                            "k_block_p2<float>, the two chunked launches of one solve as one interval"),
                        (2, "exact block solves of all levels: k_block_p1 + k_block_p2 (blocks > 1024 "
                            "cells) or k_block_dense (smaller blocks), one interval per solve"),
                        (1, "k_sweep_p<float> (finest level)")):
        H.kernel_timing(which)
        for _ in range(2):
            flush.fill_(3.0)
            step()
        launches, tot_ms, bytes_per, moved_per = H.kernel_timing_read()
        H.kernel_timing(0)
        achieved = bytes_per / (tot_ms / launches) / 1e6 if launches else None   # GB/s
        roofs[which] = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                        "unit": "GB/s", "frac": achieved / peak if achieved else None,
                        "traffic": TRAFFIC.get(which), "peak_source": src,
                        "intervals_per_solve": launches / 2, "ms_per_solve": tot_ms / 2,
                        "us_per_interval": 1e3 * tot_ms / launches,
                        "bytes_per_interval": bytes_per, "moved_bytes_per_interval": moved_per,
                        "moved_gbs": moved_per / (tot_ms / launches) / 1e6 if launches else None,
                        "note": "achieved = algorithmic bytes / event time; the working set stays in "
                                "L2 within a solve (a 1024^2 FP32 level is 12 MB); the events in the "
                                "graph serialise the launches, so ms_per_solve exceeds the kernels' "
                                "share of an untimed solve"}
    # the exact block solves take most of the solve's time (every level); the
    # roofline line reports the finest level's, whose two launches the ncu
    # capture in profiles/ covers
    roof = roofs[3]
    roof_other = roofs[1]
    roof_blocks = roofs[2]

    # plain FP64 solve of the same problem, timed like the mixed arm
    H64 = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                default_options(min_coarse_n=a.min_coarse, cycle=2, precision=0,
                                                max_cycles=60, w_depth=W_DEPTH, nu1=NU, nu2=NU))
    u64 = torch.zeros(n * n, dtype=torch.float64, device=dev)
    for _ in range(a.warmup):
        u64.zero_()
        H64.solve(ft, gt, u64, TOL, stream)
        flush.fill_(4.0)
    torch.cuda.synchronize()
    ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(a.steps)]
    for k in range(a.steps):
        flush.fill_(float(k))
        u64.zero_()
        ev64[k][0].record(stream)
        r64 = H64.solve(ft, gt, u64, TOL, stream)
        ev64[k][1].record(stream)
    torch.cuda.synchronize()
    fp64_ms = sum(s_.elapsed_time(e_) for s_, e_ in ev64) / a.steps
    err64 = float(np.abs(u64.cpu().numpy().reshape(n, n) - ue)[present].max())
    H64.close()

    # the whole cycle against HBM: the algorithmic bytes of one cycle on the
    # paper-literal one-pass-per-operation schedule, times the cycles of a
    # solve, over the device-timed solve
    blk = roof_blocks["bytes_per_interval"] * roof_blocks["intervals_per_solve"]
    roof_cycle = {f"disk_{n}": cycle_roofline(H, dof, cycles[-1], ms, peak, src,
                                              block_bytes_per_solve=blk)}

    # several independent solves at once: clones of the hierarchy (shared
    # tables, own work arrays), each with its own right-hand side, advanced
    # together by cc_solve_batch; their kernels overlap on the device
    from paper_2601_02975_gb300 import solve_batch
    nb = a.batch
    batch = None
    if nb > 0:
        hs = [H] + [H.clone(stream) for _ in range(nb - 1)]
        rng = np.random.default_rng(7)
        fb = [torch.tensor((f * (1.0 + 0.25 * rng.standard_normal())).ravel(), dtype=torch.float64,
                           device=dev) for _ in range(nb)]
        gb = [gt] * nb
        ub = [torch.zeros(n * n, dtype=torch.float64, device=dev) for _ in range(nb)]
        solve_batch(hs, fb, gb, ub, [TOL] * nb)          # warm-up (graph capture per clone)
        bms = []
        for _ in range(3):
            for x in ub:
                x.zero_()
            flush.fill_(5.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            res = solve_batch(hs, fb, gb, ub, [TOL] * nb)
            bms.append((time.perf_counter() - t) * 1e3)
            assert all(r.status == 0 for r in res)
        bms = min(bms)
        batch = {"problems": nb, "workload": f"{nb} solves of the {n}x{n} disk problem with different "
                                            "right-hand sides, one cc_solve_batch call",
                 "ms": bms, "dof_per_s": nb * dof / (bms / 1e3),
                 "vs_one_at_a_time": (nb * dof / (bms / 1e3)) / value,
                 "cycles": [r.cycles for r in res], "timing": "host wall clock around the call "
                 "(the call returns when every result is in place)"}

    serving = run_serving(a, dev) if a.serve > 0 else None
    roof_hbm = hbm_sweep(a, dev, peak, src) if a.hbm_n > 0 else None
    ellipse = run_ellipse_union(a, dev) if a.ellipse_union else None
    random_domains = run_random_domains(a, dev) if a.random_domains > 0 else None
    mcgs = run_mcgs(a, dev) if a.mcgs else None
    setup = run_setup(a, dev) if a.setup else None
    serving_full = run_serving_full(a, dev) if a.serve_full > 0 else None
    plain = run_plain_poisson(a, dev) if a.plain else None
    refine = run_refinement_sweep(a, dev) if a.plain else None
    table8 = run_table8(a, dev) if a.plain else None

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline()
    out = {
        "metric": "solved DOF/s at discretization-error accuracy (rel. residual < 1e-13)",
        "value": value, "unit": "DOF/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 cycles + f64 refinement",
        "data": "synthetic (manufactured solution exp(x)cos(2y), seeded geometry)",
        "config": {"workload": f"disk domain, (a,b,c)=(1,0.5,2), Dirichlet box + Neumann circle, "
                               f"{n}x{n} cells", "n": n, "dof_per_gpu": dof,
                   "cycle": f"W({NU},{NU}), gamma = 2 on the {W_DEPTH} finest level(s)",
                   "levels": [H.info.level_n[l] for l in range(H.info.n_levels)],
                   "precision": "mixed", "tol": TOL, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}", "cycles_per_solve": cycles[-1],
                   "autotuned": {"sweep_ctas": [H.info.sweep_ctas[l] for l in range(H.info.n_levels)],
                                 "block_chunk_rows": [H.info.block_chunk_rows[l]
                                                      for l in range(H.info.n_levels)]}},
        "e2e": {"value": e2e, "unit": "DOF/s", "h2d_bytes_per_step": 8 * (2 * n * n + H.info.n_g),
                "d2h_bytes_per_step": 8 * n * n},
        "gpu_launches": kernels,
        "roofline": roof,
        "roofline_other": roof_other,
        "roofline_blocks": roof_blocks,
        "roofline_hbm": roof_hbm,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "max_error_vs_exact": err,
        "batch": batch,
        "serving": serving,
        "ellipse_union": ellipse,
        "random_domains": random_domains,
        "multicolour_smoother": mcgs,
        "setup": setup,
        "serving_full": serving_full,
        "plain_poisson": plain,
        "refinement_sweep": refine,
        "table8_rates": table8,
        "fp64_solve": {"ms": fp64_ms, "dof_per_s": dof / (fp64_ms / 1e3), "cycles": r64.cycles,
                       "max_error_vs_exact": err64, "steps": a.steps, "warmup": a.warmup,
                       "timing": "CUDA events around each solve, L2 flushed between steps, as the "
                                 "mixed arm"},
        "roofline_cycle": roof_cycle,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
def cycle_roofline(H, dof, cycles, solve_ms, peak, src, w=4, block_bytes_per_solve=None):
    """HBM roofline of the whole solve at cycle granularity.  Algorithmic bytes
    of one FP32 cycle on the paper-literal schedule (one pass per operation):
    on every visit of a level, each of the nu1 + nu2 sweeps reads u and b and
    writes u (3 w per cell), the residual restriction reads u and b and writes
    the coarse residual (2.25 w), the prolongation reads u and the coarse
    correction and writes u (2.25 w); W(nu,nu) with gamma = 2 on the finest
    level visits it once and every coarser level twice; the bottom solve reads
    its FP64 inverse (8 n_c^2 bytes); the FP64 refinement step reads u and b
    and writes r (20 B per cell) and adds the correction (20 B).  The exact
    block solves add the method's bytes measured by cc_kernel_timing (banded
    factors plus gather).  The fused schedule of temporally blocked sweeps
    would need about 35 B per DOF per V(3,3) cycle instead."""
    import torch  # noqa: F401  (device timing done by the caller)
    info = H.info
    nl = info.n_levels
    ns = [info.level_n[l] for l in range(nl)]
    per_cycle = 0.0
    for l in range(nl - 1):
        visits = 1 if l == 0 else 2
        per_cycle += visits * ns[l] ** 2 * w * (3 * (NU + NU) + 2.25 + 2.25)
    per_cycle += 2 * 8.0 * ns[-1] ** 4                 # bottom: the dense FP64 inverse, twice
    per_cycle += 40.0 * ns[0] ** 2                     # FP64 residual and update
    per_cycle += block_bytes_per_solve / max(1, cycles)
    achieved = per_cycle * cycles / (solve_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": src, "bytes_per_cycle": per_cycle, "bytes_per_dof_per_cycle": per_cycle / dof,
            "cycles": cycles, "solve_ms": solve_ms, "levels": ns,
            "note": "paper-literal one-pass schedule, W(%d,%d) with gamma = 2 on the finest level; "
                    "FP32 cycle bytes, FP64 refinement" % (NU, NU)}


def block_bytes_per_solve(H, run):
    """Algorithmic bytes of all exact block solves of one solve (run() does one
    solve), from cc_kernel_timing."""
    H.kernel_timing(2)
    run()
    launches, tot_ms, bytes_per, moved_per = H.kernel_timing_read()
    H.kernel_timing(0)
    return launches * bytes_per


# ---------------------------------------------------------------------------
def hbm_sweep(a, dev, peak, src):
    """The finest-level FP32 sweep where it streams from HBM: two cycles of a
    Poisson solve on the unit square at hbm_n^2 (levels too large for L2),
    timed with CUDA events around each launch inside the solve graph."""
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I
    import workloads as W
    P = W.problem_poisson_square()
    n = a.hbm_n
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=1,
                                              max_cycles=2, w_depth=W_DEPTH, nu1=NU, nu2=NU))
    f, g, _ = I.problem_inputs(H, P)
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device=dev)
    gt = torch.tensor(g, dtype=torch.float64, device=dev)
    u = torch.zeros(n * n, dtype=torch.float64, device=dev)
    H.solve(ft, gt, u, 1e-300)
    H.kernel_timing(1)
    u.zero_()
    H.solve(ft, gt, u, 1e-300)
    launches, tot_ms, bytes_per, moved_per = H.kernel_timing_read()
    H.kernel_timing(0)
    H.close()
    achieved = bytes_per / (tot_ms / launches) / 1e6
    return {"kernel": f"k_sweep_p<float> (finest level, Poisson unit square {n}x{n})", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": 190.9e6 if n == 4096 else None, "peak_source": src, "launches": launches,
            "us_per_launch": 1e3 * tot_ms / launches, "bytes_per_launch": bytes_per,
            "note": "algorithmic bytes 3 x 4 x N^2 (u, b read; u written); each interval includes "
                    "the launch latency"}


def run_ellipse_union(a, dev):
    """The ellipse-union workload at 2048^2 and 4096^2: FP32 cycles in FP64
    refinement against the plain FP64 solve, both to 1e-10 relative residual
    (the accuracy floor at these sizes: the max-norm error against the exact
    cell averages no longer falls for tighter tolerances).  The FP64
    hierarchy is a clone from the setup cache, so host setup runs once."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import Hierarchy, cache_clear, default_options
    from paper_2601_02975_gb300 import inputs as I
    import workloads as W
    P = W.problem_ellipses(0)
    out = {"workload": "unit square minus ellipse union seed 0, Robin (1, 0.5), (a,b,c)=(1.5,-0.8,1), "
                       "u = sin(3x) exp(y), tol 1e-10"}
    for n in a.ellipse_union:
        row = {}
        for prec, name in ((1, "mixed"), (0, "fp64")):
            t = time.perf_counter()
            H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                      default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=prec,
                                                      max_cycles=80, w_depth=W_DEPTH, nu1=NU, nu2=NU, cache=1))
            setup = time.perf_counter() - t
            f, g, ue = I.problem_inputs(H, P)
            present = H.cell_types()[0] != 0
            ft = torch.tensor(f.ravel(), dtype=torch.float64, device=dev)
            gt = torch.tensor(g, dtype=torch.float64, device=dev)
            u = torch.zeros(n * n, dtype=torch.float64, device=dev)
            H.solve(ft, gt, u, 1e-10)
            ms = []
            for _ in range(2):
                u.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r = H.solve(ft, gt, u, 1e-10)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            err = float(np.abs(u.cpu().numpy().reshape(n, n) - ue)[present].max())
            row[name] = {"ms": min(ms), "dof_per_s": H.info.n_dof / (min(ms) / 1e3), "cycles": r.cycles,
                         "status": r.status, "rel_res": r.rel_res, "max_error_vs_exact": err,
                         "setup_s": setup}
            row["dof"] = int(H.info.n_dof)
            if prec == 1:
                def one():
                    u.zero_()
                    H.solve(ft, gt, u, 1e-10)
                peaks, src = _peaks()
                row["roofline_cycle"] = cycle_roofline(
                    H, int(H.info.n_dof), r.cycles, min(ms), float(peaks["hbm_gbs"]), src,
                    block_bytes_per_solve=block_bytes_per_solve(H, one))
            H.close()
        out[str(n)] = row
    cache_clear()
    return out


def _event_solve(H, ft, gt, u, tol, reps=3):
    """min over reps of CUDA-event time of H.solve from u = 0 (after one
    untimed solve); returns (ms, result)."""
    import torch
    u.zero_()
    H.solve(ft, gt, u, tol)
    best, r = None, None
    for _ in range(reps):
        u.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = H.solve(ft, gt, u, tol)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best, r


def _inputs(H, P, dev):
    import torch
    from paper_2601_02975_gb300 import inputs as I
    f, g, ue = I.problem_inputs(H, P)
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device=dev)
    gt = torch.tensor(g, dtype=torch.float64, device=dev)
    return ft, gt, ue


def run_plain_poisson(a, dev):
    """The plain-method case: Poisson on the unit square, u = sin(pi x)
    sin(pi y), Dirichlet, FP64 V(3,3) cycles to the coarsest level 4^2 (the
    paper's cycle) until the relative residual is below 1e-10, at 64^2;
    then the same problem at 1024^2 and 4096^2 for throughput, with the
    headline's cycle (W(4,4), gamma = 2 on the finest level, coarsest 32^2),
    FP64 and mixed."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options
    import workloads as W
    P = W.problem_poisson_square()
    out = {"workload": "Poisson, unit square, u = sin(pi x) sin(pi y), Dirichlet, tol 1e-10 "
                       "(1e-8 at 4096^2: the Dirichlet data are 0, so |b| = |f| ~ 2 pi^2 and the "
                       "relative residual of the FP64 iterate cannot fall below ~1.5e-9 there)"}
    runs = [(64, "fp64_V33", dict(min_coarse_n=4, cycle=1, precision=0, nu1=3, nu2=3))]
    for n in (1024, 4096):
        for prec, name in ((0, "fp64_W44"), (1, "mixed_W44")):
            runs.append((n, name, dict(min_coarse_n=MIN_COARSE, cycle=2, precision=prec,
                                       w_depth=W_DEPTH, nu1=NU, nu2=NU)))
    for n, name, opt in runs:
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, default_options(max_cycles=100, **opt))
        ft, gt, ue = _inputs(H, P, dev)
        u = torch.zeros(n * n, dtype=torch.float64, device=dev)
        tol = 1e-8 if n >= 4096 else 1e-10
        ms, r = _event_solve(H, ft, gt, u, tol)
        err = float(np.abs(u.cpu().numpy().reshape(n, n) - ue).max())
        out.setdefault(str(n), {})[name] = {"tol": tol,
            "ms": ms, "dof_per_s": n * n / (ms / 1e3), "cycles": r.cycles,
            "rate_per_cycle": r.rel_res ** (1.0 / max(1, r.cycles)), "max_error_vs_exact": err,
            "status": r.status, "levels": [H.info.level_n[l] for l in range(H.info.n_levels)]}
        H.close()
    return out


def run_refinement_sweep(a, dev):
    """The plain method on the irregular domain: the headline disk problem in
    FP64 (W(4,4), gamma = 2 on the finest level) to 1e-13 at 128^2 ... 1024^2,
    the max-norm and L1 errors against the exact cell averages and the
    observed order log2(e(2h)/e(h))."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options
    P = _problem()
    rows = []
    for n in (128, 256, 512, 1024):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                  default_options(min_coarse_n=MIN_COARSE if n > 128 else 16, cycle=2,
                                                  precision=0, w_depth=W_DEPTH, nu1=NU, nu2=NU,
                                                  max_cycles=80))
        ft, gt, ue = _inputs(H, P, dev)
        present = H.cell_types()[0] != 0
        u = torch.zeros(n * n, dtype=torch.float64, device=dev)
        ms, r = _event_solve(H, ft, gt, u, TOL)
        e = np.abs(u.cpu().numpy().reshape(n, n) - ue)[present]
        rows.append({"n": n, "dof": int(H.info.n_dof), "ms": ms, "dof_per_s": H.info.n_dof / (ms / 1e3),
                     "cycles": r.cycles, "rel_res": r.rel_res, "linf": float(e.max()),
                     "l1": float(e.sum()) / (n * n)})
        H.close()
    for k in range(1, len(rows)):
        rows[k]["order_linf"] = math.log2(rows[k - 1]["linf"] / rows[k]["linf"])
        rows[k]["order_l1"] = math.log2(rows[k - 1]["l1"] / rows[k]["l1"])
    return {"workload": "disk domain, (a,b,c)=(1,0.5,2), Dirichlet box + Neumann circle, "
                        "u = exp(x)cos(2y), FP64, tol 1e-13", "rows": rows}


# printed averaged residual-reduction rates (Table 8): V and FMG cycles at
# (nu1, nu2) = (2,1), (2,2), (3,3); the panda rows are out of scope
TABLE8 = {
    "unit_square": {"V": (0.858, 0.410, 0.330), "FMG": (0.672, 0.246, 0.131)},
    "rotated_square": {"V": (0.474, 0.266, 0.216), "FMG": (0.376, 0.162, 0.103)},
    "flower": {"V": (0.384, 0.318, 0.221), "FMG": (0.296, 0.207, 0.108)},
    "four_disks_D": {"V": (0.298, 0.236, 0.161), "FMG": (0.292, 0.120, 0.063)},
    "four_disks_N": {"V": (0.373, 0.336, 0.279), "FMG": (0.347, 0.208, 0.135)},
}


def run_table8(a, dev):
    """Averaged residual-reduction rates (rel. residual ^ (1 / cycles), from
    u = 0 to 1e-10) of FP64 V-cycles and FMG cycles (Alg. 3 with V) at
    (nu1, nu2) = (2,1), (2,2), (3,3) on the paper's domains at h = 1/256
    (384 cells across the rotated square's box of side 1.5), beside the
    printed values.  The paper does not state the depth of its cycles; these go
    down to the coarsest level the holes allow (at least 8^2)."""
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options
    import workloads as W
    probs = {"unit_square": (W.problem_table3(), 256, {"min_coarse_n": 64}),
             "rotated_square": (W.problem_rotated_square(), 384, {"min_coarse_n": 48}),
             "flower": (W.problem_flower(), 256, {"eps": 0.02, "min_coarse_n": 64}),
             "four_disks_D": (W.problem_four_disks(W.DIRICHLET), 256, {"eps": 0.08, "min_coarse_n": 64}),
             "four_disks_N": (W.problem_four_disks(W.NEUMANN), 256, {"eps": 0.08, "min_coarse_n": 64})}
    out = {"note": "ours / printed; FP64; three levels (the paper's depth is not stated); NaN: diverged"}
    for key, (P, n, extra) in probs.items():
        row = {}
        for cyc, cname in ((1, "V"), (3, "FMG")):
            vals = []
            for (nu1, nu2) in ((2, 1), (2, 2), (3, 3)):
                H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                          default_options(cycle=cyc, precision=0, nu1=nu1, nu2=nu2,
                                                          max_cycles=200, **extra))
                ft, gt, _ = _inputs(H, P, dev)
                u = torch.zeros(n * n, dtype=torch.float64, device=dev)
                try:
                    r = H.solve(ft, gt, u, 1e-10)
                    rate = r.rel_res ** (1.0 / max(1, r.cycles))
                except Exception as e:   # a diverging cycle is reported as such
                    rate = float("nan")
                vals.append(rate)
                H.close()
            row[cname] = {"ours": vals, "printed": list(TABLE8[key][cname])}
        out[key] = row
    return out


def run_setup(a, dev):
    """Setup time of the headline disk problem (1024^2) and of the 4096^2
    ellipse union, with the per-cell steps (classification, Def. 4.1 kinds,
    lattices, fits, curve-order samples) as CUDA kernels and on host threads;
    the two must give the same tables, bit for bit (checked on the finest
    level).  Wall clock around cc_setup; the split comes from cc_info."""
    import numpy as np
    from paper_2601_02975_gb300 import Hierarchy, default_options
    import workloads as W
    out = {"host_threads": os.cpu_count(), "cpu_model": _cpu_model()}
    for name, P, n in (("disk_1024", _problem(), a.n), ("ellipses0_4096", W.problem_ellipses(0), 4096)):
        row = {}
        tabs = []
        for d, key in ((1, "device"), (0, "host")):
            t = time.perf_counter()
            H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                      default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=1,
                                                      w_depth=W_DEPTH, nu1=NU, nu2=NU, device_setup=d))
            wall = time.perf_counter() - t
            info = H.info
            row[key] = {"s": wall, "tables_s": info.setup_tables_seconds,
                        "other_s": info.setup_seconds - info.setup_tables_seconds,
                        "kernel_ms": info.setup_kernel_ms}
            _, lat, beta = H.level_tables(0)
            tabs.append((H.cell_types()[1].copy(), lat.copy(), beta.view(np.uint64).copy(),
                         H.level_block(0).copy()))
            row["plg_cells"] = int(info.n_plg)
            H.close()
        row["tables_equal"] = all(np.array_equal(x, y) for x, y in zip(*tabs))
        row["tables_speedup"] = row["host"]["tables_s"] / row["device"]["tables_s"]
        out[name] = row
    return out


def run_mcgs(a, dev, nu=2):
    """The headline problem (1024^2 disk, mixed precision, W cycles with gamma
    = 2 on the finest level, tol 1e-13) with the multicolour Gauss-Seidel
    variant of the smoother (outside the paper; omega 0.6, nu1 = nu2 = 2,
    15 colour classes since b != 0), timed like the main arm."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import SMOOTHER_MCGS, Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I
    P = _problem()
    n = a.n
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=a.min_coarse, cycle=2, precision=1, max_cycles=80,
                                              w_depth=W_DEPTH, nu1=nu, nu2=nu, smoother=SMOOTHER_MCGS,
                                              omega=0.6))
    f, g, ue = I.problem_inputs(H, P)
    present = H.cell_types()[0] != 0
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device=dev)
    gt = torch.tensor(g, dtype=torch.float64, device=dev)
    u = torch.zeros(n * n, dtype=torch.float64, device=dev)
    for _ in range(2):
        u.zero_()
        r = H.solve(ft, gt, u, TOL)
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        u.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = H.solve(ft, gt, u, TOL)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    err = float(np.abs(u.cpu().numpy().reshape(n, n) - ue)[present].max())
    dof = int(H.info.n_dof)
    H.close()
    return {"workload": f"the headline disk problem at {n}x{n}, mixed, W({nu},{nu}) with gamma = 2 on the "
                        "finest level, multicolour smoother (15 classes, omega 0.6), tol 1e-13",
            "ms": min(ms), "dof_per_s": dof / (min(ms) / 1e3), "cycles": r.cycles, "status": r.status,
            "rel_res": r.rel_res, "kernels": r.kernels, "max_error_vs_exact": err}


def run_random_domains(a, dev):
    """Independent problems of the batch workload (random domains, operators,
    conditions and right-hand sides, N log-uniform in 64..1024), FP32 cycles
    in FP64 refinement to 1e-10: solved one at a time, then all at once with
    one cc_solve_batch call (the DOF/s count the converged problems' DOF over
    the time of all).
    Problems the setup rejects (a finest-grid cut cell with a hole inside it,
    or a coarsest level too large for the dense bottom solve) are listed as
    skipped; holes of 2-5 coarse cells can give coarsest-level cut-cell rows
    of the wrong sign and make the cycle diverge, which is reported, not
    hidden.  The same problems are then solved once more, as one batch, with
    the Krylov outer iteration (`krylov`)."""
    import torch
    from paper_2601_02975_gb300 import CCError, Hierarchy, cache_clear, default_options, solve_batch
    from paper_2601_02975_gb300 import inputs as I
    import workloads as W
    hs, fs, gs, dofs, sizes, skipped, probs = [], [], [], [], [], [], []
    t = time.perf_counter()
    for k in range(a.random_domains):
        P, n = W.problem_batch(k)
        try:
            H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                      default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=1,
                                                      max_cycles=80, w_depth=W_DEPTH, nu1=NU, nu2=NU,
                                                      cache=1))
        except CCError as e:
            skipped.append({"problem": k, "n": n, "status": e.status})
            continue
        f, g, _ = I.problem_inputs(H, P)
        probs.append((P, n))
        hs.append(H)
        fs.append(torch.tensor(f.ravel(), dtype=torch.float64, device=dev))
        gs.append(torch.tensor(g, dtype=torch.float64, device=dev))
        dofs.append(int(H.info.n_dof))
        sizes.append(n)
    setup = time.perf_counter() - t
    us = [torch.zeros(n * n, dtype=torch.float64, device=dev) for n in sizes]
    tol = [1e-10] * len(hs)
    solve_batch(hs, fs, gs, us, tol)                     # warm-up (graph capture)
    for u_ in us:
        u_.zero_()
    torch.cuda.synchronize()
    t = time.perf_counter()
    single = [solve_batch([H], [f_], [g_], [u_], [1e-10])[0] for H, f_, g_, u_ in zip(hs, fs, gs, us)]
    torch.cuda.synchronize()
    seq = time.perf_counter() - t
    alone = [u_.clone() for u_ in us]
    for u_ in us:
        u_.zero_()
    torch.cuda.synchronize()
    t = time.perf_counter()
    res = solve_batch(hs, fs, gs, us, tol)
    bat = time.perf_counter() - t
    same = all(torch.equal(x, y) for x, y in zip(us, alone))
    for H in hs:
        H.close()
    ok = [r.status == 0 for r in res]
    # the same problems through the Krylov outer iteration (FGMRES preconditioned
    # by the same cycle): clones of the cached hierarchies, no second host setup
    hk = [Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=0,
                                                max_cycles=KRYLOV_MAX_CYCLES, w_depth=W_DEPTH, nu1=NU,
                                                nu2=NU, cache=1, krylov=KRYLOV))
          for P, n in probs]
    uk = [torch.zeros(n * n, dtype=torch.float64, device=dev) for n in sizes]
    solve_batch(hk, fs, gs, uk, tol)                     # warm-up (graph capture)
    for u_ in uk:
        u_.zero_()
    torch.cuda.synchronize()
    t = time.perf_counter()
    rk = solve_batch(hk, fs, gs, uk, tol)
    bk = time.perf_counter() - t
    for H in hk:
        H.close()
    cache_clear()
    okk = [r.status == 0 for r in rk]
    krylov = {"restart": KRYLOV, "preconditioner": "one FP64 cycle", "converged": sum(okk), "statuses": [r.status for r in rk],
              "cycles": [r.cycles for r in rk], "rel_res": [r.rel_res for r in rk], "batch_ms": bk * 1e3,
              "dof_per_s_batch": sum(d for d, o in zip(dofs, okk) if o) / bk}
    return {"problems": len(hs), "skipped_at_setup": skipped, "sizes": sizes, "dof": sum(dofs),
            "setup_s": setup, "one_at_a_time_ms": seq * 1e3, "batch_ms": bat * 1e3,
            "dof_per_s_one_at_a_time": sum(d for d, o in zip(dofs, ok) if o) / seq,
            "dof_per_s_batch": sum(d for d, o in zip(dofs, ok) if o) / bat,
            "converged": sum(ok), "diverged": [sizes[i] for i, r in enumerate(res) if r.status == 6],
            "statuses": [r.status for r in res], "cycles": [r.cycles for r in res],
            "single_statuses_match": [r.status for r in single] == [r.status for r in res],
            "batch_equals_one_at_a_time": same, "krylov": krylov,
            "workload": "problems 0.. of the batch generator (1-8 holes, random a,b,c, D/N/R holes, "
                        "random-Fourier f, g = 0), tol 1e-10, host wall clock"}


SERVE_SIZES = (128, 256, 512, 1024)
SERVE_WEIGHTS = (0.5 / 3, 0.5 / 3, 0.5 / 3, 0.3)   # the request mix without its 2048^2/4096^2 share


SERVE_FULL_SIZES = (128, 256, 512, 1024, 2048, 4096)
SERVE_FULL_WEIGHTS = (0.5 / 3, 0.5 / 3, 0.5 / 3, 0.30, 0.15, 0.05)


def run_serving_full(a, dev):
    """The serving workload at its specified size: a Poisson-arrival stream
    of a.serve_full requests per rate through cc_submit / cc_poll, sizes
    128^2..4096^2 (50 % spread over 128^2-512^2, 30 % 1024^2, 15 % 2048^2,
    5 % 4096^2), each on one of a.serve_domains cached ellipse-union domains
    (seeds 0.., the 2048^2/4096^2 workload's family, set up before the
    stream, 2 slots per handle, clones within a 150 GB cc_serve_budget).
    Each request's f is its domain's manufactured f plus a random multiple of
    one of 8 random-Fourier fields (16 x 16 modes, coefficients N(0,
    1/(p^2+q^2))); tol 1e-10 (1e-9 at 4096^2, near where the FP64 cycles
    stop reducing the residual on some of these domains).  The client keeps at most 20 GB of request
    buffers on the device: a request that arrives beyond that waits on the
    host, and its latency counts from its arrival.  Domains whose validation
    request fails at some size are not served.  Mixed precision at every
    rate, FP64 (a.serve_full_fp64 requests) at the lowest and the highest;
    p50 / p99 latency (arrival to completion) and DOF/s of the solved
    requests."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options, serve_budget
    from paper_2601_02975_gb300 import inputs as I
    import workloads as W
    rng = np.random.default_rng(23)
    rates = [float(x) for x in a.serve_full_rates.split(",")]
    serve_budget(150 * (1 << 30))
    w = np.array(SERVE_FULL_WEIGHTS) / sum(SERVE_FULL_WEIGHTS)
    pert = {}
    for n in SERVE_FULL_SIZES:
        x = (np.arange(n) + 0.5) / n
        S = np.array([np.sin(p * np.pi * x) for p in range(1, 17)])
        fields = []
        for _ in range(8):
            C = rng.standard_normal((16, 16)) / np.sqrt(np.add.outer(np.arange(1, 17) ** 2, np.arange(1, 17) ** 2))
            fields.append(torch.tensor((S.T @ C @ S).ravel(), dtype=torch.float64, device=dev))
        pert[n] = fields
    out = {"requests_per_rate": a.serve_full,
           "workload": "ellipse-union domains (seeds), sizes 128^2..4096^2 at 50/30/15/5 %, Poisson "
                       "arrivals, per-request random-Fourier f, tol 1e-10 (1e-9 at 4096^2), 2 slots per handle, 150 GB "
                       "clone budget, at most 20 GB of request buffers in flight"}
    cap_bytes = 20 * (1 << 30)
    for prec, name in ((1, "mixed"), (0, "fp64")):
        t0 = time.perf_counter()
        hs, base, rejected = {}, {}, []
        for d in range(a.serve_domains):
            P = W.problem_ellipses(d)
            for n in SERVE_FULL_SIZES:
                try:
                    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                              default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=prec,
                                                              max_cycles=60, w_depth=W_DEPTH, nu1=NU, nu2=NU,
                                                              serve_slots=2))
                except Exception as e:   # a domain the setup rejects at this size
                    rejected.append((d, n, str(e)[-60:]))
                    continue
                f, g, _ = I.problem_inputs(H, P)
                hs[(d, n)] = H
                base[(d, n)] = (torch.tensor(f.ravel(), dtype=torch.float64, device=dev),
                                torch.tensor(g, dtype=torch.float64, device=dev), int(H.info.n_dof))
        ok = {d for (d, n) in hs if all((d, m) in hs for m in SERVE_FULL_SIZES)}
        # warm-up and validation: one request per handle (graphs, first clone);
        # a domain whose cycle fails at some size (diverges, or stalls above
        # the tolerance in 60 cycles) is not served
        bad = set()
        for (d, n), H in hs.items():
            fb, gb, _ = base[(d, n)]
            u = torch.zeros(n * n, dtype=torch.float64, device=dev)
            rid = H.submit(fb, gb, u, 1e-9 if n >= 4096 else 1e-10)
            while True:
                st, _ = Hierarchy.poll(rid)
                if st != 9:
                    break
                time.sleep(0.0005)
            if st != 0:
                bad.add(d)
        torch.cuda.synchronize()
        ok = sorted(ok - bad)
        out.setdefault("setup", {})[name] = {"s": time.perf_counter() - t0, "domains_served": len(ok),
                                             "pairs_rejected_at_setup": len(rejected),
                                             "domains_failing_validation": sorted(bad),
                                             "examples": rejected[:4]}
        for rate in rates:
            if prec == 0 and rate not in (rates[0], rates[-1]):
                continue
            nreq = a.serve_full if prec == 1 else min(a.serve_full, a.serve_full_fp64)
            sz = rng.choice(len(SERVE_FULL_SIZES), size=nreq, p=w)
            dm = rng.choice(ok, size=nreq)
            arrive = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
            scale = rng.standard_normal(nreq) * 20.0
            which = rng.integers(0, 8, size=nreq)
            pending, lat, dof_done, fails, held, late = {}, [], 0, {}, 0, 0
            t_start = time.monotonic()
            k = 0
            while k < nreq or pending:
                now = time.monotonic() - t_start
                while k < nreq and now >= arrive[k]:
                    n = SERVE_FULL_SIZES[sz[k]]
                    if held + 16 * n * n > cap_bytes:
                        break
                    d = int(dm[k])
                    fb, gb, ndof = base[(d, n)]
                    f = torch.add(fb, pert[n][which[k]], alpha=float(scale[k]))
                    u = torch.zeros(n * n, dtype=torch.float64, device=dev)
                    torch.cuda.current_stream(dev).synchronize()
                    late += now - arrive[k] > 0.001
                    rid = hs[(d, n)].submit(f, gb, u, 1e-9 if n >= 4096 else 1e-10)
                    pending[rid] = (n, ndof, t_start + arrive[k], f, u)
                    held += 16 * n * n
                    k += 1
                for rid in list(pending):
                    st, r = Hierarchy.poll(rid)
                    if st == 9:
                        continue
                    n, ndof, t_arr, _, _ = pending.pop(rid)
                    held -= 16 * n * n
                    lat.append(r.t_done - t_arr)
                    if st != 0:
                        fails[f"{n}:{st}"] = fails.get(f"{n}:{st}", 0) + 1
                    else:
                        dof_done += ndof
                time.sleep(0.0002)
            wall = time.monotonic() - t_start
            lat = np.sort(np.array(lat)) * 1e3
            out.setdefault(f"{rate:g}", {})[name] = {
                "requests": nreq,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "dof_per_s": dof_done / wall, "wall_s": wall, "failed": fails,
                "submitted_late": int(late)}
        for H in hs.values():
            H.close()
        torch.cuda.synchronize()
    return out


def run_serving(a, dev):
    """Poisson-arrival stream of disk-domain solves of mixed sizes through
    cc_submit / cc_poll (continuous batching, 4 slots per size), in the mixed
    and in the FP64 mode: p50 / p99 latency (submit to completion) and DOF/s."""
    import numpy as np
    import torch
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I
    P = _problem()
    rng = np.random.default_rng(11)
    w = np.array(SERVE_WEIGHTS) / sum(SERVE_WEIGHTS)
    nreq = a.serve
    sizes = rng.choice(len(SERVE_SIZES), size=nreq, p=w)
    gaps = rng.exponential(1.0 / a.serve_rate, size=nreq)
    out = {"requests": nreq, "rate_per_s": a.serve_rate,
           "sizes": {str(n): int((sizes == i).sum()) for i, n in enumerate(SERVE_SIZES)},
           "workload": "disk domain, Poisson arrivals, random-Fourier perturbation of f per "
                       "request, tol 1e-13, 4 slots per size"}
    for prec, name in ((1, "mixed"), (0, "fp64")):
        hs, base = [], []
        for n in SERVE_SIZES:
            H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                      default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=prec,
                                                      max_cycles=60, w_depth=W_DEPTH, nu1=NU, nu2=NU, serve_slots=4))
            f, g, _ = I.problem_inputs(H, P)
            hs.append(H)
            base.append((f, torch.tensor(g, dtype=torch.float64, device=dev), int(H.info.n_dof)))
        req = []
        for k in range(nreq):
            i = sizes[k]
            n = SERVE_SIZES[i]
            x = (np.arange(n) + 0.5) / n
            pert = sum(rng.standard_normal() / (p * p + q * q) * np.outer(np.sin(q * np.pi * x),
                                                                          np.sin(p * np.pi * x))
                       for p in range(1, 9) for q in range(1, 9))
            f = torch.tensor((base[i][0] + 20.0 * pert).ravel(), dtype=torch.float64, device=dev)
            req.append((i, f, torch.zeros(n * n, dtype=torch.float64, device=dev)))
        # warm-up: one request per size (graph capture, clones)
        for i in range(len(SERVE_SIZES)):
            u = torch.zeros(SERVE_SIZES[i] ** 2, dtype=torch.float64, device=dev)
            fw = torch.tensor(base[i][0].ravel(), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            rid = hs[i].submit(fw, base[i][1], u, TOL)
            while hs[i].poll(rid)[0] == 9:
                time.sleep(0.0005)
        torch.cuda.synchronize()
        pending, lat, dof_done, fails = {}, [], 0, 0
        t0 = time.perf_counter()
        t_next = t0
        k = 0
        while k < nreq or pending:
            now = time.perf_counter()
            while k < nreq and now >= t_next:
                i, f, u = req[k]
                pending[hs[i].submit(f, base[i][1], u, TOL)] = i
                k += 1
                if k < nreq:
                    t_next += gaps[k]
            for rid in list(pending):
                st, r = Hierarchy.poll(rid)
                if st == 9:
                    continue
                i = pending.pop(rid)
                if st != 0:
                    fails += 1
                lat.append(r.t_done - r.t_submit)
                dof_done += base[i][2]
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        lat = np.sort(np.array(lat)) * 1e3
        out[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "dof_per_s": dof_done / wall, "wall_s": wall, "failed": fails}
        for H in hs:
            H.close()
    return out


def _oracle_sample(n: int):
    """Oracle solve of the same disk problem on an n x n grid (setup excluded)."""
    import numpy as np
    from oracle import discretize as D
    from oracle import multigrid as M
    P = _problem()
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=MIN_COARSE)
    d = H.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    dof = int(d.lev.present.sum())

    def solve():
        return M.solve(H, b, tol=TOL, gamma=2, w_depth=W_DEPTH, nu1=NU, nu2=NU)
    return solve, dof


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_worker(args):
    """One process of the all-cores oracle baseline: set up the oracle at
    n x n, wait for the others, solve once; returns (DOF, start, end)."""
    n, barrier = args
    solve, dof = _oracle_sample(n)
    barrier.wait()
    t0 = time.time()
    solve()
    return dof, t0, time.time()


def cpu_baseline(n=256):
    """The oracle as it stands on the host cores: one solve of a 256^2 sample
    of the same problem on one core, then nproc independent solves of it in
    nproc processes at once (the oracle's numpy/scipy work is
    single-threaded, so the cores are used by running problems side by side);
    setup excluded."""
    import multiprocessing as mp
    solve, dof = _oracle_sample(n)
    t = time.perf_counter()
    r = solve()
    dt = time.perf_counter() - t
    ncore = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        bar = man.Barrier(ncore)
        with ctx.Pool(ncore) as pool:
            res = pool.map(_oracle_worker, [(n, bar)] * ncore)
    wall = max(e for _, _, e in res) - min(s_ for _, s_, _ in res)
    multi = sum(d for d, _, _ in res) / wall
    return {"value": multi, "unit": "DOF/s", "cores": ncore, "kind": "oracle",
            "cpu_model": _cpu_model(), "nproc": ncore,
            "sample": f"{ncore} FP64 oracle W({NU},{NU}) solves (gamma = 2 on the {W_DEPTH} finest "
                      f"level(s)) of the same disk problem at {n}x{n}, one per process, side by "
                      f"side ({wall:.1f} s wall); setup excluded; BLAS threads pinned to 1",
            "single_core": {"value": dof / dt, "unit": "DOF/s", "cores": 1,
                            "sample": f"one solve at {n}x{n} ({len(r.history)} cycles, {dt:.1f} s)"}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 128
    solve, dof = _oracle_sample(n)
    for _ in range(a.warmup):
        solve()
    ts = []
    for _ in range(a.steps):
        t = time.perf_counter()
        solve()
        ts.append(time.perf_counter() - t)
    ms = 1e3 * sum(ts) / len(ts)
    value = dof / (ms / 1e3)
    out = {"impl": "reference",
           "metric": "solved DOF/s at discretization-error accuracy (rel. residual < 1e-13)",
           "value": value, "unit": "DOF/s", "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"disk domain, (a,b,c)=(1,0.5,2), sample at {n}x{n} cells "
                                  f"of the {N_GRID}x{N_GRID} workload", "n": n},
           "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                            "sample": f"FP64 oracle W({NU},{NU}) solves (gamma = 2 on the {W_DEPTH} finest level(s)) at {n}x{n}, setup excluded"},
           "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile_sweep(a):
    import torch

    import __graft_entry__
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from paper_2601_02975_gb300 import inputs as I
    import workloads as W
    __graft_entry__.build()
    P = W.problem_poisson_square()
    n = a.profile_sweep
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=MIN_COARSE, cycle=2, precision=1, max_cycles=1,
                                              w_depth=W_DEPTH, nu1=NU, nu2=NU, use_graphs=0))
    f, g, _ = I.problem_inputs(H, P)
    ft = torch.tensor(f.ravel(), dtype=torch.float64, device="cuda")
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    r = H.solve(ft, gt, u, 1e-300)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "one cycle", "n": n, "cycles": r.cycles, "kernels": r.kernels}))


def main():
    a = _args()
    if a.profile_sweep:
        run_profile_sweep(a)
    elif a.profile:
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    # the oracle's numpy/scipy work runs on one thread
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    main()
