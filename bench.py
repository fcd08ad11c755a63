#!/usr/bin/env python
"""Throughput of the FP64 FD-MP5 update on GB300 (one JSON line on stdout).

Workload (the configuration the metric is quoted on): 3D ideal MHD+GLM blast,
256^3 cells as 16^3 blocks, gamma 5/3, periodic, SSPRK3, CFL 0.3, seeded
1e-3 density noise. One step = the CFL time step plus one full SSPRK3 step
(speeds, 3 x (flux pass + stage combination)) through amrfd_step_cfl; metric =
cell-updates/s, one cell-update being one full step of one active interior cell.

Arms:
  default           this library (C ABI -> CUDA kernels), N ranks = N independent
                    replicas of the workload (weak scaling, no collective).
  --impl reference  the CPU oracle (oracle/, single-threaded C, -O2), timed on the
                    host on a bounded sample (a 64^3 blast domain per step).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BLAST, BLOCK = 256, 16
NV = 9
# Algorithmic HBM bytes per cell-update (SSPRK3, nv = 9): stage reads/writes of
# U^n, U^(k) and the output, (2 + 3 + 3) * nv * 8 = 64 nv = 576 bytes.
BYTES_PER_CELL_UPDATE = 64 * NV
# Minimal HBM bytes of one flux pass per cell: read U^(k) (nv doubles) and write
# the three per-direction residuals (3 nv doubles). The kernel also reads five
# derived quantities per cell (40 B), traffic spent to save FP64 work.
FLUX_BYTES_PER_CELL = 4 * NV * 8
# FP64 work of the flux pass per cell and direction (flop = DADD + DMUL + 2 DFMA thread
# instructions, counted by ncu on the 128^3 blast's first step, 32 lines per tile, with a
# build whose sums and products were still DADD and DMUL; the kernels now issue them as
# FMAs by 1 and with -0, the same instruction count, which 2 x DFMA no longer reads as flop):
# 291.96 at 16-cell segments, 273.17 at 32-cell segments. A segment of S cells computes
# the split flux of its S + 6 cells and starts its sweeps afresh, so the count is
# a + b/S; the method's own work (one split flux per cell, one reconstruction per face,
# no segment overheads) is the limit a = 254.4 of the two measurements. Of b = 601.3,
# 6 x 57 flop is the halo's split flux (the MHD+GLM flux along one direction, 21 flop,
# and its split, 18 FMAs) and 259.3 the sweep restart (the extra face and the opening
# differences), which a segment swept in parts pays per part.
FLUX_FLOPS_PER_CELL_DIR = 254.4
FLUX_FLOP_HALO = 6 * 57.0
FLUX_FLOP_SWEEP_START = 259.3


def flux_flop_executed(seg, part):
    """FP64 flop per cell and direction the flux pass executes with segments of seg cells
    swept in parts of part cells."""
    return FLUX_FLOPS_PER_CELL_DIR + FLUX_FLOP_HALO / seg + FLUX_FLOP_SWEEP_START / part


FP64_PEAK_TFLOPS_NOMINAL = 1.25   # GB300 FP64, nominal (context only)
# DRAM bytes per cell of one flux launch (ncu dram__bytes_read + write of the 128^3 blast's
# first flux pass, tile 64 x 8 lines x 320 threads, scaled by cells): traffic grows with
# the cells processed
FLUX_TRAFFIC_BYTES_PER_CELL = (443.714560 + 413.586944) * 1e6 / 128 ** 3


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def clocks_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def clocks_summary(path, gpu_index):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms_local, cells_per_rank, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: the slowest rank's time over
    the units all ranks processed. Returns (ms_max, cell-updates/s)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, cells_per_rank * steps * world / (ms_max * 1e-3)


def cpu_baseline(cells_side=128, block=16):
    """The oracle as it stands: one SSPRK3 step of an n^3 blast on one host core."""
    import oracle as O
    from paper_1407_2052_gb300 import workloads as W
    w = W.blast3d(cells_side, block)
    d0 = w.domains[0]
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    od = O.dom(d0.n, d0.dx, bc=[list(b) for b in d0.bc], nb=d0.nb)
    h, _ = O.dt(c, od, w.U, w.cfl)
    t0 = time.perf_counter()
    h, _ = O.dt(c, od, w.U, w.cfl)
    O.step(c, od, w.U, h)
    el = time.perf_counter() - t0
    return {"value": cells_side ** 3 / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "one CFL dt + one SSPRK3 step of the %d^3 blast (%d^3 blocks), %.1f s" % (cells_side, block, el)}


def batched_extra(torch, A, W, steps=2):
    """20000 uneven independent blocks, 30% passive: persistent work-list launches
    (graph) vs one launch per domain (block) per pass, both with the flux tile the
    autotuner picks for this work; active cell-updates/s."""
    w = W.batched(20000)
    s = A.Solver.from_workload(w)
    ncell_active = sum(d.ncell for d, a in zip(w.domains, w.active) if a)
    U0 = torch.from_numpy(w.U).cuda()
    del w
    U = U0.clone()
    dt = torch.empty(s.ndom, dtype=torch.float64, device="cuda")
    tile_default = list(s.get_tile())
    s.dt(U, out=dt)
    t0 = time.perf_counter()
    tile = list(s.autotune(U, dt))
    out = {"workload": "20000 blocks, edges {8,12,16,24,32}^3, 30% passive, MHD+GLM SSPRK3",
           "active_cells": ncell_active, "tile": tile, "tile_default": tile_default,
           "autotune_s": time.perf_counter() - t0}
    for name, fn in (("persistent", s.step_batched), ("per_block", s.step)):
        U.copy_(U0)
        s.dt(U, out=dt)
        fn(U, dt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            s.dt(U, out=dt)
            fn(U, dt)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "cell_updates_per_s": ncell_active / (ms * 1e-3)}
    assert s.error() == A.OK
    out["speedup"] = out["per_block"]["ms_per_step"] / out["persistent"]["ms_per_step"]
    s.close()
    del U, U0
    torch.cuda.empty_cache()
    return out


def adjoint_extra(torch, A, W, reps=3):
    """2D MHD+GLM 512^2, fixed dt 1e-3, SSPRK3: one adjoint step vs one forward step, both
    with the flux tile the autotuner picks for the forward step."""
    w = W.adjoint2d(512)
    s = A.Solver.from_workload(w)
    U = torch.from_numpy(w.U.ravel().copy()).cuda()
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    tile = list(s.autotune(U, dt))
    g = torch.randn(U.numel(), dtype=torch.float64, device="cuda")
    gout = torch.empty_like(U)
    V = U.clone()
    s.step_batched(V, dt)
    s.adjoint(U, dt, g, gout)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        V.copy_(U)
        s.step_batched(V, dt)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        s.adjoint(U, dt, g, gout)
    e1.record()
    torch.cuda.synchronize()
    adj = e0.elapsed_time(e1) / reps
    # the full gradient: 200 steps with checkpoints every 20 (forward, recomputation and
    # adjoints) against 200 forward steps
    from paper_1407_2052_gb300 import autodiff
    area = w.domains[0].dx[0] * w.domains[0].dx[1]
    e0.record()
    V.copy_(U)
    for _ in range(200):
        s.step_batched(V, dt)
    e1.record()
    torch.cuda.synchronize()
    fwd200 = e0.elapsed_time(e1)
    # three gradients: the first also captures the step graphs of the rollout's buffers and
    # allocates them; each is split into forward run, recomputation and adjoint steps
    runs = []
    for _ in range(3):
        U0r = U.clone().requires_grad_(True)
        stats = {}
        torch.cuda.synchronize()
        e0.record()
        Uf = autodiff.rollout(s, U0r, dt, 200, 20, stats=stats)
        B = Uf.view(9, -1)[5:8]
        (0.5 * (B * B).sum() * area).backward()
        e1.record()
        torch.cuda.synchronize()
        stats["gradient_ms"] = e0.elapsed_time(e1)
        runs.append(stats)
        grad = U0r.grad.detach().clone()
        del U0r, Uf, B
    grad200 = min(r["gradient_ms"] for r in runs)
    # for information: central differences (h = 1e-6) of the actual 200-step GPU run along 4
    # seeded unit directions, the splitting speeds recomputed from the perturbed states (the
    # adjoint holds them at their forward values: the map with speeds recomputed differs)
    gen = torch.Generator(device="cuda").manual_seed(14072052)
    hfd, worst = 1e-6, 0.0
    gnorm = float(grad.norm())

    def final_B(U):
        Vb = U.clone()
        for _ in range(200):
            s.step_batched(Vb, dt)
        return Vb.view(9, -1)[5:8]
    for _ in range(4):
        v = torch.randn(U.numel(), dtype=torch.float64, device="cuda", generator=gen)
        v /= v.norm()
        Bp, Bm = final_B(U + hfd * v), final_B(U - hfd * v)
        fd = float(0.5 * ((Bp - Bm) * (Bp + Bm)).sum() * area / (2 * hfd))
        worst = max(worst, abs(fd - float((grad * v).sum())) / gnorm)
    assert s.error() == A.OK
    s.close()
    return {"workload": "adjoint2d: 2D MHD+GLM 512^2, SSPRK3, dt 1e-3", "tile": tile, "forward_ms": fwd, "adjoint_ms": adj,
            "ratio": adj / fwd, "rollout_200_steps_every_20": {"forward_ms": fwd200, "gradient_ms": grad200,
                                                                 "ratio": grad200 / fwd200, "runs": runs,
                                                                 "unfrozen_fd_rel_discrepancy": worst,
                                                                 "unfrozen_fd": "4 directions, h 1e-6, relative "
                                                                 "to the gradient's norm"}}


def _time_steps(torch, fn, steps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def schemes_extra(torch, A, W, tile, steps=2):
    """Cost of one step of the blast (256^3 in 16^3 blocks) under the paper's scheme
    pairings (Sec. 4.5.2 times SSPRK(5,4)-MP5 against RK3-LIMO3 at 2.2 : 1)."""
    w = W.blast3d(256, 16)
    U0 = torch.from_numpy(w.U.ravel()).cuda()
    out = {"workload": "blast3d 256^3 in 16^3 blocks, MHD+GLM, dt from CFL 0.3 of U^0"}
    for name, integ, recon in (("ssprk54_mp5", A.SSPRK54, A.MP5), ("ssprk3_mp5", A.SSPRK3, A.MP5),
                               ("rk3_limo3", A.SSPRK3, A.LIMO3)):
        s = A.Solver(w.physics, w.ndim, integ, w.gamma, w.cfl, w.domains, active=w.active, glm_cr=w.glm_cr,
                     recon=recon)
        s.set_tile(*tile)
        U = U0.clone()
        dt = s.dt(U)
        ms = _time_steps(torch, lambda: s.step_batched(U, dt), steps)
        assert s.error() == A.OK
        out[name] = {"ms_per_step": ms, "cell_updates_per_s": w.domains[0].ncell / (ms * 1e-3)}
        s.close()
        del U
    out["ratio_ssprk54_mp5_to_rk3_limo3"] = out["ssprk54_mp5"]["ms_per_step"] / out["rk3_limo3"]["ms_per_step"]
    del U0
    torch.cuda.empty_cache()
    return out


def activation_extra(torch, A, W, tile, steps=3):
    """Dynamic grid activation (App. C) on the quiet blast (uniform background), 256^3 in
    16^3 blocks: criterion |U - U_background| <= 1e-12, a two-block belt and the device
    work-list rebuild before every step, against all blocks active. Early in the run most
    of the box is still at rest, so most blocks are passive."""
    import numpy as np
    w = W.blast3d(256, 16, noise=0.0)
    U0 = torch.from_numpy(w.U.ravel()).cuda()
    R = torch.from_numpy(w.extra["background"].ravel()).cuda()
    ncell = w.domains[0].ncell
    out = {"workload": "quiet blast3d 256^3 in 16^3 blocks, MHD+GLM SSPRK3, belt 2, first steps"}
    for mode in ("all_active", "dynamic"):
        s = A.Solver.from_workload(w)
        U = U0.clone()
        dt = torch.empty(1, dtype=torch.float64, device="cuda")
        flag = torch.empty(s.nblocks, dtype=torch.uint8, device="cuda")
        s.set_tile(*tile)

        def one():
            if mode == "dynamic":
                s.activate(s.flag_steady(U, R, 1e-12, out=flag), 2)
            s.dt(U, out=dt)
            s.step_batched(U, dt)
        ms = _time_steps(torch, one, steps)
        used = list(tile)
        if mode == "dynamic":
            # segments through several blocks skip less where few blocks are active: the
            # sparse work list also timed with one-block segments, the faster kept
            U.copy_(U0)
            s.set_tile(16, 32, 288)
            ms16 = _time_steps(torch, one, steps)
            if ms16 < ms:
                ms, used = ms16, [16, 32, 288]
        assert s.error() == A.OK
        frac = float(s.active().float().mean().item())
        out[mode] = {"ms_per_step": ms, "active_block_fraction": frac,
                     "domain_cells_per_s": ncell / (ms * 1e-3), "tile": used}
        s.close()
        del U
    out["speedup"] = out["all_active"]["ms_per_step"] / out["dynamic"]["ms_per_step"]
    del U0, R
    torch.cuda.empty_cache()
    # the paper's main gain from passive blocks: a larger global CFL step. 20000 uneven
    # blocks with one global dt; the finest tenth (smallest dx) handed to another
    # treatment (passive, belt 0): dt grows by the ratio of the limiting cell sizes
    w = W.batched(20000)
    s = A.Solver.from_workload(w, dt_scope=A.DT_GLOBAL)
    U = torch.from_numpy(w.U).cuda()
    dx = np.array([d.dx[0] for d in w.domains])
    flag = torch.from_numpy((dx < np.quantile(dx, 0.1)).astype(np.uint8) | (1 - w.active)).cuda()
    del w
    res = {}
    for mode in ("all", "fine_passive"):
        if mode == "fine_passive":
            s.activate(flag, 0)
        dt = s.dt(U)
        h = float(dt[0].item())
        ms = _time_steps(torch, lambda: s.step_batched(U, dt), 2)
        res[mode] = {"dt": h, "ms_per_step": ms, "simulated_time_per_s": h / (ms * 1e-3)}
    assert s.error() == A.OK
    res["dt_gain"] = res["fine_passive"]["dt"] / res["all"]["dt"]
    res["simulated_time_rate_gain"] = res["fine_passive"]["simulated_time_per_s"] / res["all"]["simulated_time_per_s"]
    out["global_dt_batched"] = res
    s.close()
    del U
    torch.cuda.empty_cache()
    return out


def full_run_extra(torch, A, W, tile, nsteps=200):
    """The whole 200-step blast (256^3 in 16^3 blocks, SSPRK3, CFL 0.3) from U^0, one CUDA
    event per step: the cost of the early steps (the window the headline times) against the
    late ones, when the blast has spread and the limiter works at more faces."""
    w = W.blast3d(256, 16)
    s = A.Solver.from_workload(w)
    s.set_tile(*tile)
    U = torch.from_numpy(w.U.ravel()).cuda()
    ncell = w.domains[0].ncell
    del w
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
    torch.cuda.synchronize()
    ev[0].record()
    for i in range(nsteps):
        s.step_cfl(U, out=dt)
        ev[i + 1].record()
    torch.cuda.synchronize()
    assert s.error() == A.OK
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(nsteps)]

    def rate(a, b):
        m = sum(ms[a:b]) / (b - a)
        return {"steps": "%d-%d" % (a + 1, b), "ms_per_step": m, "cell_updates_per_s": ncell / (m * 1e-3)}
    out = {"workload": "blast3d 256^3 in 16^3 blocks, MHD+GLM SSPRK3, CFL 0.3, %d steps from U^0" % nsteps,
           "all": rate(0, nsteps), "early_6_25": rate(5, 25), "late_181_200": rate(nsteps - 20, nsteps)}
    out["late_over_early"] = out["late_181_200"]["ms_per_step"] / out["early_6_25"]["ms_per_step"]
    s.close()
    del U
    torch.cuda.empty_cache()
    return out


def workload_config(nside):
    """The workload both arms report on (the reference arm times a bounded sample of it)."""
    return {"workload": "blast3d: 3D ideal MHD+GLM blast, %d^3 cells in 16^3 blocks, SSPRK3, CFL 0.3" % nside,
            "cells": nside ** 3, "integrator": "SSPRK3"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as O
    from paper_1407_2052_gb300 import workloads as W
    n = 64
    w = W.blast3d(n, BLOCK)
    d0 = w.domains[0]
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    od = O.dom(d0.n, d0.dx, bc=[list(b) for b in d0.bc], nb=d0.nb)
    U = w.U.copy()
    for _ in range(args.warmup):
        h, _ = O.dt(c, od, U, w.cfl)
        U, _, _, _ = O.step(c, od, U, h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h, _ = O.dt(c, od, U, w.cfl)
        U, _, _, _ = O.step(c, od, U, h)
    el = time.perf_counter() - t0
    val = n ** 3 * args.steps / el
    sample = ("each step: one CFL dt + one SSPRK3 step of the same blast at %d^3 (%d^3 blocks) on one host "
              "core, the oracle's cell-updates/s standing for the %d^3 run" % (n, BLOCK, args.n))
    out = {"metric": "3D MHD FD-MP5 cell-updates/s (FP64)", "value": val, "unit": "cell-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": dict(workload_config(args.n), parallelism="single host core",
                          sample_cells=n ** 3),
           "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch

    import __graft_entry__ as g
    from paper_1407_2052_gb300 import amrfd as A
    from paper_1407_2052_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    g.build()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    nside = args.n
    w = W.blast3d(nside, BLOCK)
    ncell = nside ** 3
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel()).cuda()
    U = U0.clone()
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    del w

    def one_step():
        # CFL dt of U^n and one SSPRK3 step, the speed maxima of U^n shared
        s.step_cfl(U, out=dt)

    def one_step_graph():
        s.dt(U, out=dt)
        s.step_batched(U, dt)

    tile_default = list(s.get_tile())
    if args.tile:
        s.set_tile(*[int(x) for x in args.tile.split(",")])
    elif not args.no_autotune:
        s.dt(U, out=dt)
        s.autotune(U, dt)
    for _ in range(args.warmup):
        one_step()
    UW = U.clone()          # state at the start of the timed region
    barrier()

    # ---- timed region: K steps, CUDA events around every kernel (same stream)
    gpu_index = local_rank
    try:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            gpu_index = int(vis.split(",")[local_rank])
    except ValueError:
        pass
    import tempfile
    clk_dir = args.clocks_dir or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, "clocks_bench_rank%d.csv" % rank)
    proc, fh = clocks_sampler(clk_path)
    s.timing_begin(16 * args.steps + 16)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    barrier()
    kt = s.timing_end()
    ms = e0.elapsed_time(e1)
    if proc is not None:
        proc.terminate()
        proc.wait()
        fh.close()
    clocks = clocks_summary(clk_path, gpu_index)
    assert s.error() == A.OK
    ms_max, value = aggregate(ms, ncell, args.steps, world, dist, "cuda")
    launches = sum(v[1] for v in kt.values())
    Uend = U.clone()

    # ---- the same K steps as amrfd_dt + the step replayed from its captured CUDA graph
    U.copy_(UW)
    for _ in range(2):
        one_step_graph()
    U.copy_(UW)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        one_step_graph()
    e1.record(stream)
    barrier()
    graph_ms = e0.elapsed_time(e1) / args.steps

    # ---- end to end through the public API with host buffers (pinned): every step uploads
    # its input state host -> device and downloads its result device -> host, and the next
    # step of that trajectory uploads the downloaded result. NT trajectories take turns, each
    # starting from the state the timed region had at its first step of that trajectory, so
    # that together they take exactly the K steps timed above; while one computes, the
    # others' copies run on an upload and a download stream.
    NT = min(3, args.steps)
    starts = [(args.steps * i + NT - 1) // NT for i in range(NT + 1)]   # step index of each start
    U.copy_(UW)
    first = []
    for i in range(args.steps):
        if i in starts[:NT]:
            first.append(U.clone())
        one_step()
    hst = [torch.empty(U.shape, dtype=U.dtype).pin_memory() for _ in range(NT)]
    nbytes = hst[0].numel() * 8
    bufs = [U] + [torch.empty_like(U) for _ in range(NT - 1)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()   # host->device, device->host
    dts = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in range(NT)]
    ev_in = [torch.cuda.Event() for _ in range(NT)]
    ev_out = [torch.cuda.Event() for _ in range(NT)]
    ev_free = [torch.cuda.Event() for _ in range(NT)]
    lens = [starts[i + 1] - starts[i] for i in range(NT)]

    def e2e_steps(lengths):
        done = [0] * NT
        i = 0
        while any(done[b] < lengths[b] for b in range(NT)):
            b = i % NT
            i += 1
            if done[b] >= lengths[b]:
                continue
            with torch.cuda.stream(up):
                if done[b] > 0:
                    up.wait_event(ev_free[b])      # the trajectory's previous result is home
                bufs[b].copy_(hst[b], non_blocking=True)
                ev_in[b].record(up)
            stream.wait_event(ev_in[b])
            s.step_cfl(bufs[b], out=dts[b])
            ev_out[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_out[b])
                hst[b].copy_(bufs[b], non_blocking=True)
                ev_free[b].record(down)
            done[b] += 1
        stream.wait_stream(up)
        stream.wait_stream(down)

    for b in range(NT):
        hst[b].copy_(first[b])
    e2e_steps([1] * NT)
    torch.cuda.synchronize()
    # this box's pinned copy rates for the state (the e2e figure hides them behind compute
    # unless a copy takes longer than the other trajectories' steps)
    rates = {}
    for name, dst, src in (("h2d_gbs", bufs[-1], hst[0]), ("d2h_gbs", hst[0], bufs[-1])):
        best = 1e30
        for _ in range(3):
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        rates[name] = nbytes / (best * 1e-3) / 1e9
    for b in range(NT):
        hst[b].copy_(first[b])
    clk2_path = os.path.join(clk_dir, "clocks_e2e_rank%d.csv" % rank)
    proc2, fh2 = clocks_sampler(clk2_path)
    barrier()
    e0.record(stream)
    e2e_steps(lens)
    e1.record(stream)
    barrier()
    if proc2 is not None:
        proc2.terminate()
        proc2.wait()
        fh2.close()
    e2e_clocks = clocks_summary(clk2_path, gpu_index)
    # each trajectory ends where the next began; the last where the timed region ended
    for b in range(NT - 1):
        assert torch.equal(hst[b], first[b + 1].cpu())
    assert torch.equal(hst[NT - 1], Uend.cpu())
    e2e_ms = e0.elapsed_time(e1)
    _, e2e_value = aggregate(e2e_ms, ncell, args.steps, world, dist, "cuda")

    flux_ms, flux_n = kt["flux"]
    flux_avg_s = flux_ms / max(flux_n, 1) * 1e-3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # the FP64 rate this GPU sustains, measured here (the flux pass runs inside a long step)
    fp64 = A.fp64_peak(seconds=2.0)
    seg_eff = min(int(s.get_tile()[0]), nside)
    part_eff = seg_eff // (seg_eff // 16) if seg_eff >= 32 else seg_eff
    achieved = FLUX_FLOPS_PER_CELL_DIR * 3 * ncell / flux_avg_s / 1e12
    executed = flux_flop_executed(seg_eff, part_eff) * 3 * ncell / flux_avg_s / 1e12
    roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved, "peak": fp64["sustained_tflops"],
            "frac": achieved / fp64["sustained_tflops"], "traffic": FLUX_TRAFFIC_BYTES_PER_CELL * ncell,
            "kernel": "flux_kernel", "launch_ms": flux_avg_s * 1e3,
            "flop_per_cell_dir": FLUX_FLOPS_PER_CELL_DIR,
            "flop_per_cell_dir_executed": flux_flop_executed(seg_eff, part_eff),
            "executed_tflops": executed, "executed_frac": executed / fp64["sustained_tflops"],
            "peak_source": "measured: amrfd_fp64_peak, independent FP64 FMAs on every SM, back to back for 2 s "
                           "(sustained); burst %.3f TFLOP/s" % fp64["burst_tflops"],
            "peak_nominal": FP64_PEAK_TFLOPS_NOMINAL}
    flux_gbs = FLUX_BYTES_PER_CELL * ncell / flux_avg_s / 1e9
    out = {
        "metric": "3D MHD FD-MP5 cell-updates/s (FP64)",
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(nside), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (%.2f GB state)" % (ncell * NV * 8 / 1e9), "tile": list(s.get_tile()),
                   "tile_default": tile_default, "autotuned": not (args.no_autotune or args.tile)},
        "gpu_launches": launches,
        "kernel_ms": {k: {"total": v[0], "launches": v[1]} for k, v in kt.items()},
        "graph_ms_per_step": graph_ms,
        "roofline": roof,
        "roofline_hbm": {"bound": "hbm", "unit": "GB/s",
                         "achieved_step": value / world * BYTES_PER_CELL_UPDATE / 1e9,
                         "achieved_flux": flux_gbs, "peak": hbm_peak,
                         "frac_step": value / world * BYTES_PER_CELL_UPDATE / 1e9 / hbm_peak,
                         "frac_flux": flux_gbs / hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                         "frac_step_of_nominal_7900": value / world * BYTES_PER_CELL_UPDATE / 1e9 / 7900.0},
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes,
                "note": "pinned host buffers; the K timed steps as three trajectories taking turns, each "
                        "step uploading its trajectory's last downloaded result; copies on two streams "
                        "overlap the other trajectories' compute",
                "clocks": e2e_clocks, "h2d_gbs": rates["h2d_gbs"], "d2h_gbs": rates["d2h_gbs"]},
        "clocks": clocks,
    }
    tile = list(s.get_tile())
    s.close()
    del U, U0, UW, Uend, bufs, hst, first
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras:
        out["batched"] = batched_extra(torch, A, W)
        out["adjoint"] = adjoint_extra(torch, A, W)
        out["schemes"] = schemes_extra(torch, A, W, tile)
        out["activation"] = activation_extra(torch, A, W, tile)
        out["full_run"] = full_run_extra(torch, A, W, tile)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched-block and adjoint comparisons")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default flux-pass tile")
    ap.add_argument("--tile", default="", help="seg,lines,threads of the flux pass (skips autotuning)")
    ap.add_argument("--n", type=int, default=N_BLAST, help="cells per side of the blast (profiling of small cases)")
    ap.add_argument("--clocks-dir", default="", help="where to keep the nvidia-smi clock samples (default: temp dir)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
