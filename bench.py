#!/usr/bin/env python
"""Benchmark: FGMRES solve time and apply GB/s at relative residual 1e-8, mixed precision
vs FP64, with step-latency percentiles, on one GB300 (replicas on N GPUs).

Workload (the configuration the headline metric is quoted on): Carreau Stokes
(nu0 = 1, nu_inf = 1e-3, lambda = 1, n = 0.5, frozen Picard velocity from seed 2) in a
32x32x32-element Q2/Q1 channel with four cylindrical obstacles, 4x4x4 subdomains grouped
2x2x2, three-level monolithic GDSW, FGMRES(100) to 1e-8.  Synthetic seeded inputs.

One step = one Picard linear solve: Carreau viscosity at the Gauss points and re-assembly
of the saddle-point operator, the lifted right-hand side, and the GDSW-preconditioned
FGMRES solve (every row of the hot path).  The preconditioner factors are built once
before timing.  Inputs (factors: 15 GB FP32) are far larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gdsw|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "channel32_4cyl_carreau_n0.5_q2q1_4x4x4_grouped2x2x2_3level"
DIE_WORKLOAD = "die64x64x128_sdf_carreau_n0.4_q2q1_rcb512_64_8_4level"
METRIC = "FGMRES solve time and apply GB/s at rel res 1e-8, mixed vs FP64; p99 latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gdsw", "reference"], default="gdsw")
    ap.add_argument("--mixed", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison context")
    ap.add_argument("--m", type=int, default=32, help="elements per edge of the channel")
    ap.add_argument("--workload", choices=["channel", "die", "mg"], default="channel",
                    help="channel: 32^3 Carreau channel (3 levels); die: 64x64x128 die-like channel (4 levels); "
                         "mg: geometric multigrid on the 64^3 Carreau cube with its 16^3 grid solved by 4-level GDSW")
    ap.add_argument("--pressure", choices=["q1", "p1disc"], default="q1",
                    help="channel workload: Q2/Q1 (default) or the Q2/P1-disc pair")
    ap.add_argument("--levels", type=int, default=0,
                    help="channel workload: 2 or 3 levels (0: 3 for Q2/Q1, 2 for Q2/P1-disc)")
    ap.add_argument("--mg-m", type=int, default=64, help="elements per edge of the finest multigrid grid")
    ap.add_argument("--mg-smoother", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--mg-nu", type=int, default=3, help="pre- and post-smoothing steps")
    ap.add_argument("--mg-symmetric", type=int, default=1, help="1: post-smoothing in reverse colour order")
    ap.add_argument("--mg-restart", type=int, default=200)
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--prof-stride", type=int, default=1,
                    help="CUDA-event timing of every k-th preconditioner apply in the profiled pass")
    ap.add_argument("--sweep", choices=["auto", "persistent", "steps"], default="auto",
                    help="local solves: the set-up autotuner's choice, one persistent launch per level, "
                         "or one launch per slab step")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="resident CTAs per SM of the persistent sweep (0 = all)")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per forward GEMV tile (0 = the autotuner's)")
    ap.add_argument("--graph", type=int, default=0, help="1: the preconditioner apply replays a captured CUDA graph")
    ap.add_argument("--serve", action="store_true", help="serving workload: Poisson arrivals of mixed requests")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--serve-sizes", type=str, default="8,12,16,20,24,28,32")
    ap.add_argument("--slots", type=int, default=8)
    return ap.parse_args()


def gemv_traffic_ratio(persistent):
    """DRAM bytes / algorithmic bytes of the level-1 sweep from the committed ncu summary of
    that kernel, valid only while the kernel source is the one that was profiled (else None)."""
    import hashlib
    name = "k_sweep_channel32_dram.json" if persistent else "k_gemv_channel32_dram.json"
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2606_01433_gb300", "csrc", "dense.cu")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return d["dram_over_algorithmic"] if d.get("dense_cu_sha256") == sha else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "0x1") or v == "Active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("GDSW_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def allreduce_max(v, world, device=None):
    """Max over ranks (replicas: the slowest rank defines the job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle
GOLDEN = os.path.join(ROOT, "tests", "golden", "channel32_oracle.json")


def oracle_iterations(p):
    """The oracle's own FGMRES iteration count on this workload (to 1e-8), from the golden
    file that tests/golden/make_channel32_oracle.py writes with oracle/ alone."""
    d = json.load(open(GOLDEN))
    assert d["workload"] == p.name and d["tol"] == 1e-8, "golden file is for another workload"
    return int(d["iterations"]), d


def oracle_sample(p):
    """cpu_baseline: the FP64 oracle, as it stands, on a bounded sample of the workload, on
    a pool of all host cores (oracle/parallel.py), scaled to ms per step.  Sample: the full
    assembly (pool threads), the factorisation of one level-1 subdomain per worker (spread
    over the size range; set-up, excluded) and one parallel round of their local solves, one
    SpMV; per step = assembly + its x (64/W rounds of local solves + SpMV), with the
    oracle's own iteration count its (golden file).  Coarse levels, Phi products and the
    Arnoldi work are left out of this sample; the reference arm times them."""
    import numpy as np
    from oracle import fem, gdsw as og
    from oracle.parallel import HostPool
    its, _ = oracle_iterations(p)
    with HostPool() as pool:
        t0 = time.perf_counter()
        S = fem.assemble(p, pool=pool)
        t_asm = time.perf_counter() - t0
        A = S["A"]
        dofs = og.overlapping_dofs(S, p)
        order = np.argsort([len(d) for d in dofs], kind="stable")
        pick = order[np.unique(np.linspace(0, len(dofs) - 1, min(pool.cores, len(dofs))).round().astype(int))]
        pool.share_csr("A", A)
        pool.factor("sample", "A", [dofs[i] for i in pick])
        r = np.random.default_rng(0).standard_normal(A.shape[0])
        pool.solve("sample", r)
        t0 = time.perf_counter()
        pool.solve("sample", r)
        t_round = time.perf_counter() - t0
        pool.matvec(A, r)
        t0 = time.perf_counter()
        pool.matvec(A, r)
        t_spmv = time.perf_counter() - t0
        cores = pool.cores
    rounds = len(dofs) / len(pick)
    ms = 1e3 * (t_asm + its * (rounds * t_round + t_spmv))
    sample = ("oracle on a pool of %d host cores: full assembly (%.2f s); one parallel round of %d level-1 "
              "subdomain solves (%.1f ms, x%.1f rounds per apply) + one SpMV (%.1f ms) per iteration, x%d oracle "
              "iterations; factorisations excluded (set-up), coarse levels, Phi products and Arnoldi not sampled"
              % (cores, t_asm, len(pick), 1e3 * t_round, rounds, 1e3 * t_spmv, its))
    return ms, sample, cores


def oracle_reference(p, steps, warmup):
    """Reference arm: the complete FP64 oracle on a pool of all host cores.

    Set-up (timed once, reported apart): assembly, the multilevel GDSW set-up and one
    complete GDSW-FGMRES solve to 1e-8, which gives the oracle's own iteration count and its
    Arnoldi/least-squares time.  Each step is a bounded sample: one complete preconditioner
    apply (every level) and one SpMV of the oracle, timed; ms per step = assembly +
    iterations x (apply + SpMV) + the solve's remaining Krylov work."""
    import numpy as np
    from oracle import fem, fgmres, gdsw as og
    from oracle.parallel import HostPool
    with HostPool() as pool:
        t0 = time.perf_counter()
        S = fem.assemble(p, pool=pool)
        t_asm = time.perf_counter() - t0
        t0 = time.perf_counter()
        P = og.GDSW(S, p, pool=pool)
        t_setup = time.perf_counter() - t0
        A = S["A"]
        b = fem.lifted_rhs(S)
        acc = {"apply": 0.0, "spmv": 0.0}

        def timed(key, fn):
            def run(v):
                t = time.perf_counter()
                out = fn(v)
                acc[key] += time.perf_counter() - t
                return out
            return run
        t0 = time.perf_counter()
        x, info = fgmres.fgmres(timed("spmv", lambda v: pool.matvec(A, v)), b, timed("apply", P.apply),
                                tol=1e-8, restart=100, max_it=1000)
        t_solve = time.perf_counter() - t0
        its = info["iterations"]
        t_rest = t_solve - acc["apply"] - acc["spmv"]
        rng = np.random.default_rng(0)
        vals = []
        wall0 = time.perf_counter()
        for k in range(warmup + steps):
            r = rng.standard_normal(A.shape[0])
            t0 = time.perf_counter()
            P.apply(r)
            t_a = time.perf_counter() - t0
            t0 = time.perf_counter()
            pool.matvec(A, r)
            t_s = time.perf_counter() - t0
            if k >= warmup:
                vals.append(1e3 * (t_asm + its * (t_a + t_s) + t_rest))
        wall = time.perf_counter() - wall0
        cores = pool.cores
    return {"ms": statistics.mean(vals), "cores": cores, "iterations": its, "relres": info["relres"],
            "assembly_s": t_asm, "setup_s": t_setup, "full_solve_s": t_solve, "krylov_rest_s": t_rest,
            "apply_s_mean": acc["apply"] / max(its, 1), "spmv_s_mean": acc["spmv"] / max(its + 2, 1),
            "sample_wall_s": wall}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores (the reference arm)."""
    if rank != 0:
        return
    from paper_2606_01433_gb300 import inputs as I
    p = I.channel(args.m)
    o = oracle_reference(p, args.steps, args.warmup)
    v = o["ms"]
    sample = ("complete oracle set-up and one complete solve to 1e-8 (%d iterations, %.1f s, assembly %.1f s) on a "
              "pool of %d host cores; per step one complete oracle preconditioner apply + one SpMV, timed, scaled "
              "by the oracle's iteration count, plus the assembly and the solve's remaining Krylov work"
              % (o["iterations"], o["full_solve_s"], o["assembly_s"], o["cores"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.m == 32 else WORKLOAD.replace("channel32", "channel%d" % args.m),
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": o["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle": {k: o[k] for k in ("iterations", "relres", "assembly_s", "setup_s", "full_solve_s",
                                         "krylov_rest_s", "apply_s_mean", "spmv_s_mean", "sample_wall_s")},
            "measured_complete_step_ms": 1e3 * (o["assembly_s"] + o["full_solve_s"])}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- serving
def run_serving(n_req, sizes, slots, seed=5, budget_frac=0.8, fixed_rate=False, closed_req=None):
    """Continuous batching of mixed Carreau requests (unit-cube channels m^3, m ~ U{sizes},
    n ~ U[0.3, 1], nu0/nu_inf log-uniform in [10, 1e4]).  Closed loop first (all submitted at
    once: throughput; on the first closed_req requests of the mix when given), then open loop
    with Poisson arrivals of all n_req requests at 0.8x that throughput (latency = submit ->
    result in host memory)."""
    import numpy as np
    import torch
    from paper_2606_01433_gb300 import gdsw, inputs as I
    reqs = I.serving_requests(n_req, seed, sizes)
    probs = [I.carreau_cube(r["m"], r["n"], r["nu_inf"], r["seed"]) for r in reqs]
    free, _ = torch.cuda.mem_get_info()
    srv = gdsw.Server(device=torch.cuda.current_device(), mem_budget_bytes=int(free * budget_frac), max_slots=slots)
    st, _ = srv.gdsw_server_wait(srv.gdsw_server_submit(probs[0]))  # warm-up
    nc = n_req if closed_req is None else min(closed_req, n_req)
    t0 = time.perf_counter()
    tickets = [srv.gdsw_server_submit(p) for p in probs[:nc]]
    closed = [srv.gdsw_server_wait(t)[0] for t in tickets]
    makespan = time.perf_counter() - t0
    thr = nc / makespan
    def open_loop(gaps):
        tickets = []
        t0 = time.perf_counter()
        due = 0.0
        for p, gap in zip(probs, gaps):
            due += gap
            delay = due - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.gdsw_server_submit(p))
        done = [srv.gdsw_server_wait(t)[0] for t in tickets]
        return done, time.perf_counter() - t0

    rng = np.random.default_rng(seed)
    opened, wall = open_loop(rng.exponential(1.0 / (0.8 * thr), size=n_req))
    fixed = None
    if fixed_rate:  # the same rate with equal gaps
        fixed, fwall = open_loop(np.full(n_req, 1.0 / (0.8 * thr)))
    stats = srv.gdsw_server_stats_read()
    srv.close()
    lat = np.array([s.latency_ms for s in opened])
    ok = sum(1 for s in closed + opened + (fixed or []) if s.state == gdsw.REQ_DONE and s.relres <= 1e-8)
    extra = {}
    if fixed:
        fl = np.array([s.latency_ms for s in fixed])
        extra = {"fixed_rate": {"rate_per_s": 0.8 * thr, "throughput_per_s": n_req / fwall,
                                "latency_ms": {"p50": float(np.percentile(fl, 50)), "p99": float(np.percentile(fl, 99)),
                                               "max": float(fl.max())}}}
    return {"requests": n_req, "sizes": list(sizes), "slots": slots, "closed_loop_solves_per_s": thr,
            "closed_loop_makespan_s": makespan, "open_loop_rate_per_s": 0.8 * thr,
            "open_loop_throughput_per_s": n_req / wall, **extra,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "setup_ms_p50": float(np.median([s.setup_ms for s in opened])),
            "solve_ms_p50": float(np.median([s.solve_ms for s in opened])),
            "queue_ms_p50": float(np.median([s.queue_ms for s in opened])),
            "iterations_p50": float(np.median([s.iterations for s in opened])),
            "closed_loop_requests": nc,
            "converged": ok, "of": nc + (2 if fixed else 1) * n_req, "peak_running": stats.peak_running,
            "peak_used_gb": stats.peak_used_bytes / 1e9, "budget_gb": stats.budget_bytes / 1e9,
            "local_precision": "fp32"}


def run_serve_mode(args, rank, world, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    sizes = tuple(int(s) for s in args.serve_sizes.split(","))
    res = run_serving(args.requests, sizes, args.slots, fixed_rate=True)
    if rank == 0:
        line = {"metric": "served Stokes solves: p50/p99 latency (ms) under Poisson arrivals at 0.8x closed-loop "
                          "throughput", "value": res["latency_ms"]["p99"], "unit": "ms", "n_gpus": world,
                "higher_is_better": False, "scaling": "weak", "dtype": "f32", "data": "synthetic",
                "config": {"workload": "serving_carreau_cubes", "requests": args.requests},
                "serving": res}
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- multigrid arm
MG_WORKLOAD = "mg_cube{m}_carreau_n0.5_q2q1_3grids_vanka_coarse_gdsw4"


def run_mg(args, rank, world, local):
    """Geometric multigrid whose coarse problem the four-level GDSW method solves (Section 3;
    configuration 4): the unit-cube Carreau channel on grids m^3, (m/2)^3, (m/4)^3; symmetric
    V(nu, nu) cycles (nu = 3 by default) with the element-Vanka smoother (FP32 patch inverses by
    default), the coarsest grid
    solved by GDSW-preconditioned FGMRES to 1e-1 (parts of 2^3 elements grouped 2x2x2 twice:
    four levels); FP64 FGMRES on the finest grid to 1e-8, preconditioned by one V-cycle per
    iteration.  One step = one solve of the seeded random right-hand side."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01433_gb300 import gdsw, inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m = args.mg_m
    q = m // 4 // 2
    probs = I.mg_hierarchy(m, 3, parts=(q, q, q), groups=((2, 2, 2), (2, 2, 2)), levels=4, seed=4)
    t0 = time.perf_counter()
    G = gdsw.Multigrid(probs, pre=args.mg_nu, post=args.mg_nu, smoother=args.mg_smoother, coarse_tol=1e-1,
                       tol=1e-8, restart=args.mg_restart, max_it=2000, symmetric=bool(args.mg_symmetric))
    setup_s = time.perf_counter() - t0
    n = G.n
    b = torch.from_numpy(I.random_rhs(n, probs[0].rhs_seed)).to(dev)
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        info = G.solve(b, x)
    st0 = G.gdsw_mg_stats()
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    lib = gdsw.load()
    launches0 = lib.gdsw_kernel_launches()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    evs[0].record(stream)
    its = []
    for k in range(args.steps):
        x.zero_()
        info = G.solve(b, x)
        its.append(info.iterations)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = lib.gdsw_kernel_launches() - launches0
    total_ms = allreduce_max(evs[0].elapsed_time(evs[-1]), world, dev)
    st1 = G.gdsw_mg_stats()
    ms = total_ms / args.steps
    cycles = (st1["cycles"] - st0["cycles"]) / args.steps
    coarse_its = (st1["coarse_iterations"] - st0["coarse_iterations"]) / max(st1["coarse_solves"] - st0["coarse_solves"], 1)
    # end to end: b from pinned host memory, x back to host, inside the timed region
    bh = torch.from_numpy(I.random_rhs(n, probs[0].rhs_seed)).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bd = bh.to(dev, non_blocking=True)
        xd = torch.zeros_like(bd)
        G.solve(bd, xd)
        xh.copy_(xd, non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = allreduce_max((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)
    sizes = [int(g.n) for g in G.grids]
    relres = info.relres
    G.close()
    if rank == 0:
        line = {"metric": "multigrid solve time at rel res 1e-8 (FP64 FGMRES, V-cycle preconditioned, GDSW coarse solver)",
                "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.mg_smoother == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": MG_WORKLOAD.format(m=m), "grids_dofs": sizes, "smoother": args.mg_smoother,
                           "cycle": "V(%d,%d)" % (args.mg_nu, args.mg_nu), "symmetric": bool(args.mg_symmetric),
                           "restart": args.mg_restart, "coarse_tol": 1e-1, "tol": 1e-8,
                           "l2": "inputs larger than L2 (no flush)"},
                "iterations": its[-1], "relres": relres, "vcycles_per_solve": cycles,
                "coarse_fgmres_iterations_mean": coarse_its, "setup_s": setup_s, "clocks": clk,
                "gpu_launches": launches,
                "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}}
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def run_gdsw(args, rank, world, local):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01433_gb300 import gdsw, inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "die":
        p = I.die()
        mixed = (args.mixed, "fp32", "fp32")
        wname = DIE_WORKLOAD
    else:
        two = args.levels == 2 or (args.pressure == "p1disc" and args.levels == 0)
        p = I.channel(args.m, groups=(), levels=2) if two else I.channel(args.m)
        p.pressure = args.pressure
        mixed = (args.mixed, args.mixed, args.mixed)
        wname = WORKLOAD if args.m == 32 else WORKLOAD.replace("channel32", "channel%d" % args.m)
        if two:
            wname = wname.replace("_grouped2x2x2_3level", "_2level")
        if args.pressure == "p1disc":
            wname = wname.replace("q2q1", "q2p1disc")
    t0 = time.perf_counter()
    ctx = gdsw.Context(p, precision=mixed, phi_precision="fp32", tol=1e-8, restart=100, max_it=1000,
                       use_graph=bool(args.graph))
    setup_mixed_s = time.perf_counter() - t0
    if args.sweep != "auto":
        ctx.gdsw_set_local_sweep(args.sweep == "persistent", args.ctas_per_sm, args.tile_rows)
    tuned = ctx.sizes
    persistent = bool(tuned.persistent[0]) if args.sweep == "auto" else args.sweep == "persistent"
    n = ctx.n
    lib = gdsw.load()
    import ctypes
    def plan_bytes(direction):
        out = []
        while True:
            d = ctypes.c_double()
            if lib.gdsw_plan_bytes(ctx.h, 0, direction, len(out), ctypes.byref(d)) != 0:
                return out
            out.append(d.value)
            if direction == 2:
                return out
    fwd_bytes, bwd_bytes, red_bytes = plan_bytes(0), plan_bytes(1), plan_bytes(2)
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)

    def step(c):
        c.gdsw_reassemble()
        c.gdsw_rhs_lift(b)
        x.zero_()
        return c.gdsw_solve(b, x)

    for _ in range(args.warmup):
        info = step(ctx)
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = Clocks(local)
    launches0 = lib.gdsw_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    if args.profile_region:
        torch.cuda.profiler.start()
    evs[0].record(stream)
    iters = []
    for k in range(args.steps):
        info = step(ctx)
        iters.append(info.iterations)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.stop()
    barrier(world)
    clk = clocks.stop()
    launches = lib.gdsw_kernel_launches() - launches0
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = allreduce_max(total_ms, world, dev)
    relres = info.relres
    # profiled pass: the same steps again with CUDA events around every kernel group of
    # every prof_stride-th apply (per-kernel times for the roofline; kept out of the headline)
    ctx.gdsw_profile_enable(args.prof_stride)
    ctx.gdsw_profile_reset()
    for _ in range(args.steps):
        step(ctx)
    torch.cuda.synchronize()
    prof = ctx.gdsw_profile_read()
    ctx.gdsw_profile_enable(False)
    fp64_tflops = gdsw.probe_fma("fp64")
    fp32_tflops = gdsw.probe_fma("fp32")
    # dominant kernel: the level-1 block-LDU sweep GEMV
    loc = prof["local"]
    gemv_gbs = loc["bytes"] / (loc["ms"] * 1e-3) / 1e9 if loc["ms"] > 0 else None
    gemv_avg_ms = loc["ms"] / max(loc["calls"], 1)
    gemv_avg_bytes = loc["bytes"] / max(loc["calls"], 1)
    ap = prof["apply"]
    apply_gbs = ap["bytes"] / (ap["ms"] * 1e-3) / 1e9 if ap["ms"] > 0 else None
    sp = prof["spmv"]
    spmv_gbs = sp["bytes"] / (sp["ms"] * 1e-3) / 1e9 if sp["ms"] > 0 else None
    ar = prof["arnoldi"]
    asm_ms = (prof["assembly"]["ms"] + prof["viscosity"]["ms"]) / args.steps
    kernels = {}
    for name, g in prof.items():
        if g["calls"] > 0 and g["ms"] > 0:
            kernels[name] = {"calls": int(g["calls"]), "ms_per_call": g["ms"] / g["calls"],
                             "bytes_per_call": g["bytes"] / g["calls"],
                             "gbs": g["bytes"] / (g["ms"] * 1e-3) / 1e9}
    sizes0 = ctx.sizes
    spmv_flops = 18.0 * sizes0.nnzb_A + 12.0 * sizes0.nnz_B
    spmv_tflops = spmv_flops / (sp["ms"] / max(sp["calls"], 1) * 1e-3) / 1e12 if sp["ms"] > 0 else None

    # FP64 path for the mixed-vs-FP64 comparison
    fp64 = None
    if not args.no_fp64:
        del ctx
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        c64 = gdsw.Context(p, precision=("fp64",) * 3, phi_precision="fp64", tol=1e-8)
        setup64 = time.perf_counter() - t0
        if args.sweep != "auto":
            c64.gdsw_set_local_sweep(args.sweep == "persistent", args.ctas_per_sm, args.tile_rows)
        for _ in range(min(args.warmup, 1)):
            step(c64)
        c64.gdsw_profile_enable(True)
        c64.gdsw_profile_reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        its64 = []
        for _ in range(args.steps):
            its64.append(step(c64).iterations)
        e1.record(stream)
        torch.cuda.synchronize()
        p64 = c64.gdsw_profile_read()
        a64 = p64["apply"]
        l64 = p64["local"]
        fp64 = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "iterations": its64[-1], "setup_s": setup64,
                "apply_gbs": a64["bytes"] / (a64["ms"] * 1e-3) / 1e9 if a64["ms"] > 0 else None,
                "apply_ms": a64["ms"] / max(a64["calls"], 1),
                "local_gemv_gbs": l64["bytes"] / (l64["ms"] * 1e-3) / 1e9 if l64["ms"] > 0 else None}
        c64.close()
        del c64
        torch.cuda.empty_cache()
        ctx = gdsw.Context(p, precision=mixed, phi_precision="fp32", tol=1e-8, use_graph=bool(args.graph))
        if args.sweep != "auto":
            ctx.gdsw_set_local_sweep(args.sweep == "persistent", args.ctas_per_sm, args.tile_rows)

    # end to end through the host-buffer entry point: u_k, b and x0 from pinned host memory,
    # x back to host, inside the timed region
    uk_h = torch.from_numpy(np.ascontiguousarray(p.uk)).pin_memory().numpy()
    ctx.gdsw_reassemble()
    ctx.gdsw_rhs_lift(b)
    b_h = b.cpu().pin_memory().numpy()
    x_h = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    ctx.gdsw_reassemble(uk_h)
    ctx.gdsw_solve_host(b_h.copy(), x_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.gdsw_reassemble(uk_h)
        x_h[:] = 0.0
        ctx.gdsw_solve_host(b_h, x_h)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = allreduce_max(e2e_ms, world, dev)
    h2d = uk_h.nbytes + b_h.nbytes + x_h.nbytes
    d2h = x_h.nbytes
    sizes = ctx.sizes
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    serving = None
    if os.environ.get("GDSW_BENCH_NO_SERVE") != "1":
        # the serving mix (256 requests of 8^3 .. 32^3, 8 slots, Poisson arrivals at 0.8x the
        # closed-loop rate measured on the first 64 requests)
        serving = run_serving(256, (8, 12, 16, 20, 24, 28, 32), 8, closed_req=64)

    peak, peak_kind = measured_peaks()
    ms_step = total_ms / args.steps
    headline = args.workload == "channel" and args.m == 32 and args.pressure == "q1" and args.levels in (0, 3)
    ratio = gemv_traffic_ratio(persistent) if (headline and args.mixed == "fp32") else None
    line = {
        "metric": METRIC,
        "value": ms_step,
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.mixed == "fp32" else "bf16",
        "data": "synthetic",
        "config": {"workload": wname, "n_dofs": n, "levels": int(sizes.levels),
                   "subdomains": [int(v) for v in list(sizes.n_parts)[:sizes.levels - 1]],
                   "coarse": [int(v) for v in list(sizes.n_coarse)[:sizes.levels - 1]],
                   "local_precision": args.mixed, "krylov_precision": "f64", "tol": 1e-8, "restart": 100,
                   "apply_graph": bool(args.graph),
                   "l2": "inputs larger than L2 (no flush)", "replicas": world},
        "iterations": iters[-1],
        "relres": relres,
        "solve_ms": ms_step - asm_ms,
        "assembly_ms": asm_ms,
        "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99)),
                       "max": max(step_ms)},
        "apply_gbs": apply_gbs,
        "apply_ms": ap["ms"] / max(ap["calls"], 1),
        "spmv_gbs": spmv_gbs,
        "spmv_fp64": {"flops_per_call": spmv_flops, "tflops": spmv_tflops, "fp64_fma_peak_tflops": fp64_tflops,
                      "frac_of_fp64_peak": (spmv_tflops / fp64_tflops) if spmv_tflops else None,
                      "frac_of_hbm": (spmv_gbs / measured_peaks()[0]) if spmv_gbs else None},
        "fma_probe_tflops": {"fp64": fp64_tflops, "fp32": fp32_tflops},
        "kernels": kernels,
        "profiled_pass": "kernel-group times from CUDA events on every %d-th apply of a second run of the same "
                         "%d steps after the timed region" % (args.prof_stride, args.steps),
        "arnoldi_ms_per_solve": ar["ms"] / max(ar["calls"], 1) * iters[-1],
        "spmv_ms_per_solve": sp["ms"] / max(sp["calls"], 1) * (iters[-1] + 2),
        "fp64": fp64,
        "speedup_vs_fp64": (fp64["ms_per_step"] / ms_step) if fp64 else None,
        "setup_s": setup_mixed_s,
        "setup_breakdown_ms": dict(zip(["host_symbolic", "viscosity_assembly", "level1_factors", "phi_and_A0",
                                        "coarse_levels", "total"], [float(v) for v in sizes.setup_ms])),
        "factor_gb": sizes.factor_entries[0] * (4 if args.mixed == "fp32" else 2) / 1e9,
        "roofline": {"kernel": ("k_sweep (level-1 persistent block-LDL^T sweep, one launch per apply)" if persistent
                                else "k_gemv/k_sym_reduce/k_gemvt (level-1 block-LDL^T sweep: one chained launch "
                                     "per slab step, the chain of one apply timed as one unit)"),
                     "bound": "hbm", "achieved": gemv_gbs,
                     "peak": peak, "unit": "GB/s", "frac": (gemv_gbs / peak) if gemv_gbs else None,
                     "peak_kind": peak_kind, "avg_launch_ms": gemv_avg_ms, "avg_launch_bytes": gemv_avg_bytes,
                     "traffic": (ratio * gemv_avg_bytes) if ratio else None,
                     "fwd_launch_bytes": fwd_bytes, "bwd_launch_bytes": bwd_bytes, "reduce_bytes": red_bytes},
        "autotune": {"tile_rows": [int(v) for v in list(tuned.tile_rows)[:tuned.levels - 1]],
                     "persistent": [int(v) for v in list(tuned.persistent)[:tuned.levels - 1]],
                     "local_solve_ms": [float(v) for v in list(tuned.tuned_ms)[:tuned.levels - 1]]},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "serving": serving,
    }
    if rank == 0:
        if world == 1 and os.environ.get("GDSW_BENCH_NO_CPU") != "1" and headline:
            ms, sample, cores = oracle_sample(p)
            line["cpu_baseline"] = {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample}
        else:
            line["cpu_baseline"] = None
        line["throughput_solves_per_s"] = world * 1e3 / ms_step
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl != "reference" and os.environ.get("GDSW_LAUNCH_OVERLAP") == "0":
        import __graft_entry__
        __graft_entry__.build()
        from paper_2606_01433_gb300 import gdsw
        gdsw.set_launch_overlap(False)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.serve:
        run_serve_mode(args, rank, world, local)
    elif args.workload == "mg":
        run_mg(args, rank, world, local)
    else:
        run_gdsw(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
