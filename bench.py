#!/usr/bin/env python
"""Benchmark of the block-forest AMR lattice Boltzmann step on one GB300.

Workload: 3D lid-driven cavity, D3Q19, FP32, 64^3 root cells in 4^3-cell
blocks, lid u = 0.05, Re = 1000, up to 3 extra levels (L_max = 4) by the
vorticity criterion, adaptation every 50 coarse steps.  One bench step = one
adaptation period: 50 coarse steps of the recursive level step (interpolate,
collide + stream, average on every level) followed by one adaptation (sync,
criterion, refine/coarsen, relink, interpolation to new children).

value   = MLUPS over the timed steps (lattice updates of leaf cells, the
          Section 5.1 definition: sum_L 2^L N_leaf_cells,L per coarse step),
          device time from CUDA events, L2 flushed before every timed step.
e2e     = the same metric through the C ABI with every step's result (rho, u
          of all blocks) copied to pinned host memory inside the timed region.
roofline= fused collide-stream kernel: algorithmic bytes 2 Q N_p per update
          over its CUDA-event time (events captured inside the coarse-step
          graph), against the measured HBM copy bandwidth.

Multi-GPU: one independent replica per rank (the instance does not shard);
value = all ranks' updates / max-over-ranks time, scaling "weak".
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PERIOD = 50
HBM_FALLBACK_GBS = 6800.0
CAVITY_WORKLOAD = ("3D lid-driven cavity D3Q19 BGK FP32, 64^3 root cells in 4^3 blocks, lid "
                   "0.05, Re 1000, L_max 4 (vorticity criterion N_start -2, N_inc 1), "
                   "adaptation every 50 coarse steps")
PAPER_A100_MLUPS = 1753.0     # paper, 3D LDC D3Q19 FP32 64^3 L_max 4 on A100 (context)

# ncu DRAM traffic of k_collide_stream<3,19,float> per cell update on the
# single-level 256^3 D3Q19 FP32 forest, and the hash of the kernel source it
# was measured on.  A changed source reports null.
NCU_TRAFFIC_PER_UPDATE = 152.2     # bytes (dram read + write) per cell update
NCU_SOURCE_SHA = "408d1e3a376e2bc2"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("collide_stream.cuh", "lattice.cuh"):
        with open(os.path.join(ROOT, "paper_2308_08085_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        import numpy as np
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------- the oracle leg
def cpu_info():
    """Host core count and CPU model (the oracle runs on these cores)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": os.uname().machine}


class OracleSample:
    """The CPU oracle, as it stands, on a bounded sample of the workload: the
    cavity of the benchmark cut to 32^3 root cells (D3Q19, the same Re 1000,
    L_max 4, vorticity criterion every 50 coarse steps; the oracle cut of the
    parity tests), spun up for 50 coarse steps and one adaptation (untimed);
    then whole coarse steps are timed until a budget of seconds has passed."""

    def __init__(self, n=32, spin_periods=1, spin_every=50):
        import workloads as W
        from oracle.solver import ForestLBM
        self.n, self.spin = n, (spin_periods, spin_every)
        self.sim = ForestLBM(W.config_c1(n=n, max_blocks=(n // 4) ** 3 * 80))
        for _ in range(spin_periods):
            self.sim.step(spin_every)
            self.sim.adapt()
        self.ups = self.sim.updates_per_coarse_step()

    def run(self, budget_s):
        t0 = time.perf_counter()
        steps = 0
        while time.perf_counter() - t0 < budget_s or steps == 0:
            self.sim.step(1)
            steps += 1
        return self.ups * steps, time.perf_counter() - t0, steps

    def describe(self):
        return ("oracle ForestLBM (numpy, FP64) on the benchmark cavity cut to %d^3 root "
                "cells (Re 1000, L_max 4) after %d coarse steps and one adaptation; "
                "coarse steps of %d leaf updates each, blocks per level %s"
                % (self.n, self.spin[0] * self.spin[1], self.ups, self.sim.mesh.counts()))


FULL_RUNS = {
    # name: (config factory, coarse steps, criterion every)
    "c0": (lambda W: W.config_c0(), 2000, 100),
    "c1cut": (lambda W: W.config_c1(n=32, max_blocks=(32 // 4) ** 3 * 80), 150, 50),
}


def oracle_full_run(name):
    """The oracle's complete run of one of FULL_RUNS: coarse steps with the
    criterion-driven adaptation every `every` steps, all of it timed."""
    import workloads as W
    from oracle.solver import ForestLBM
    mk, steps, every = FULL_RUNS[name]
    sim = ForestLBM(mk(W))
    upd = 0
    t0 = time.perf_counter()
    for _ in range(steps // every):
        upd += every * sim.updates_per_coarse_step()
        sim.step(every)
        sim.adapt()
    return upd, time.perf_counter() - t0, sim.mesh.counts()


def cpu_worker(args):
    """One process of the oracle leg: `--cpu-steps` steps of `--cpu-budget`
    seconds each, after the spin-up; prints the per-step updates and times.
    With `--cpu-run`, the complete run of FULL_RUNS[name] instead."""
    if args.cpu_run:
        u, t, counts = oracle_full_run(args.cpu_run)
        print(json.dumps({"steps": [[u, t, 1]], "desc": "blocks per level at the end %s"
                          % (counts,)}))
        return
    s = OracleSample()
    steps = []
    for _ in range(max(1, args.cpu_steps)):
        u, t, n = s.run(args.cpu_budget)
        steps.append([u, t, n])
    print(json.dumps({"steps": steps, "desc": s.describe()}))


def oracle_processes(procs, budget, n_steps, timeout, run=None):
    """Run `procs` oracle workers at once (fresh interpreters, one thread
    each); returns their JSON results.  The workers are independent replicas
    of the sample: the oracle is a plain single-threaded program."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--cpu-budget",
           str(budget), "--cpu-steps", str(n_steps)] + (["--cpu-run", run] if run else [])
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                           env=env) for _ in range(procs)]
    res = []
    for p in ps:
        try:
            out, _ = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            out = ""
        line = [l for l in out.splitlines() if l.startswith("{")]
        if p.returncode == 0 and line:
            res.append(json.loads(line[-1]))
    return res


def aggregate(res, first_step=0):
    """MLUPS of concurrent workers: all their updates over the longest
    worker's time, counting steps from `first_step` on."""
    upd = sum(sum(s[0] for s in r["steps"][first_step:]) for r in res)
    sec = max(sum(s[1] for s in r["steps"][first_step:]) for r in res)
    return upd / sec / 1e6, upd, sec


def run_cpu_baseline(budget):
    """The oracle leg of the default run: one worker (one core), then one
    worker per host core at once, `budget` seconds each."""
    info = cpu_info()
    one = oracle_processes(1, budget, 1, budget * 20 + 300)
    if not one:
        return None
    v1, u1, s1 = aggregate(one)
    n = max(1, info["nproc"] or 1)
    alln = oracle_processes(n, budget, 1, budget * 20 + 600)
    out = {"value": round(v1, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": one[0]["desc"] + "; timed %.1f s" % s1, "seconds": round(s1, 2),
           "cpu_model": info["model"], "nproc": info["nproc"], "machine": info["machine"]}
    if len(alln) == n:
        vn, un, sn = aggregate(alln)
        out["all_cores"] = {"value": round(vn, 4), "unit": "MLUPS", "cores": n,
                            "processes": n, "seconds": round(sn, 2),
                            "note": "one oracle process per core at once, each the sample "
                                    "above; all their updates over the longest time"}
    return out


# ---------------------------------------------------------------- our arm
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_ranks(dist, seconds, units, device):
    """Whole-job figures over the ranks of a replica run: the slowest rank's
    time and the units (cell updates) all ranks processed."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def run_ours(args):
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    cfg = W.config_c1(n=args.n, max_blocks=(args.n // 4) ** 3 * args.cap_factor)
    sim = AmrLBM(cfg, storage="f32", kernel_variant=args.variant)
    capacity_errors = 0
    for _ in range(args.warmup):
        sim.step(PERIOD)
        rc, _ = sim.adapt()
        capacity_errors += rc != 0
    torch.cuda.synchronize()
    start_counts = sim.counts()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sim.profile(2)
    sim.profile_read(reset=True)
    updates = 0
    launches0 = sim.counts()["launches"]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_updates = []
    active_updates = 0
    torch.cuda.nvtx.range_push("timed")            # ncu --nvtx --nvtx-include "timed/"
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                      # untimed: evict L2 between steps
        step_updates.append(PERIOD * sim.updates_per_coarse_step())
        updates += step_updates[-1]
        cnt = sim.counts()
        active_updates += PERIOD * sum((2 ** L) * cnt["n_active"][L] * sim.m
                                       for L in range(sim.lmax))
        e0, e1, e2 = ev[k]
        e0.record(stream)
        sim.step(PERIOD)
        e1.record(stream)
        rc, _ = sim.adapt()
        capacity_errors += rc != 0
        e2.record(stream)
        sim.profile_read(reset=False)              # one graph-captured coarse-step sample
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = sim.counts()["launches"] - launches0     # this library's kernels only
    t_total = sum(e0.elapsed_time(e2) for e0, _, e2 in ev) / 1e3
    # windows of two timed steps (100 coarse steps each, adaptation included)
    win = [(step_updates[i] + step_updates[i + 1])
           / ((ev[i][0].elapsed_time(ev[i][2]) + ev[i + 1][0].elapsed_time(ev[i + 1][2])) / 1e3)
           / 1e6 for i in range(0, args.steps - 1, 2)]
    t_solver = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / 1e3
    prof = sim.profile_read(reset=True)
    sim.profile(0)
    end_counts = sim.counts()
    leaf_updates_end = sim.updates_per_coarse_step()   # the mesh of the last timed step

    t_max, upd_all = combine_ranks(dist, t_total, updates, dev)

    # end to end through the C ABI: result fields to pinned host memory
    nbytes = sim.field_bytes(0)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    import ctypes
    e2e_updates = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_updates += PERIOD * sim.updates_per_coarse_step()
        sim.step(PERIOD)
        sim.adapt()
        rc = sim.lib.amr_fields(sim.h, 0, ctypes.c_void_p(host.data_ptr()), nbytes, 0)
        assert rc == nbytes
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    t_e2e, e2e_updates = combine_ranks(dist, t_e2e, e2e_updates, dev)

    # the paper's steady-state figure (Section 5.1): the mean over the last
    # samples of the instantaneous MLUPS of single coarse steps, each timed
    # alone (solver only; the mesh adapts every PERIOD coarse steps, untimed)
    inst = []
    section51_start = sim.counts()["coarse_steps"]
    if args.paper_samples > 0:
        ev1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.paper_samples)]
        ups_k = []
        for k in range(args.paper_samples):
            if k % PERIOD == 0:
                sim.adapt()
                ups = sim.updates_per_coarse_step()
            ups_k.append(ups)
            ev1[k][0].record(stream)
            sim.step(1)
            ev1[k][1].record(stream)
        torch.cuda.synchronize()
        inst = [u / (a.elapsed_time(b) / 1e3) / 1e6 for u, (a, b) in zip(ups_k, ev1)]

    # roofline of the fused collide-stream kernel
    cs = prof.get("collide_stream", {})
    peak, peak_kind = measured_peaks()
    roof = None
    if cs.get("ms", 0) > 0:
        achieved = cs["bytes"] / (cs["ms"] / 1e3) / 1e9
        per_launch_updates = cs["cells"] / max(1, cs["launches"])
        traffic = None
        if NCU_TRAFFIC_PER_UPDATE is not None and NCU_SOURCE_SHA == kernel_source_sha():
            traffic = round(NCU_TRAFFIC_PER_UPDATE * per_launch_updates)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_kind + " hbm_gbs (MEASURED_PEAKS.json copy test)",
                "kernel": "k_collide_stream<3,19,float>",
                "bytes_per_update": 2 * 19 * 4,
                "sampled_launches": cs["launches"],
                "avg_launch_ms": round(cs["ms"] / max(1, cs["launches"]), 5),
                "avg_updates_per_launch": round(per_launch_updates, 1)}
    # every profiled kernel kind over the sampled coarse steps: time share and
    # achieved algorithmic bandwidth (interpolation: 2^D parent cells per child
    # with ghost cells read + ghost cells written; averaging: interface fine
    # cells read + one parent cell per 2^D written)
    step_kinds = {k: v for k, v in prof.items() if not k.startswith("adapt_")}
    t_prof = sum(v["ms"] for v in step_kinds.values()) or 1.0
    share = {k: {"ms": round(v["ms"], 4), "share": round(v["ms"] / t_prof, 4),
                 "launches": v["launches"],
                 "gbs": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                 "frac": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / peak, 4) if v["ms"] > 0 else None}
             for k, v in step_kinds.items()}
    # phases of the timed adaptations (device time between phase events)
    adapt_phases = {k[len("adapt_"):]: round(v["ms"] / max(1, v["launches"]), 4)
                    for k, v in prof.items() if k.startswith("adapt_") and v["launches"]}

    # single-level periodic 256^3 D3Q19 FP32 forest: the stencil's roofline bar
    bar = None
    if not args.no_bar:
        del flush
        bar = {order: run_bar(args, AmrLBM, W, torch, dev, stream, order)
               for order in ("lexicographic", "morton", "shuffled")}

    out = None
    if rank == 0:
        value = upd_all / t_max / 1e6
        out = {
            "metric": "MLUPS", "value": round(value, 2), "unit": "MLUP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": round(value / PAPER_A100_MLUPS, 3),
            "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": CAVITY_WORKLOAD,
                "step": "50 coarse steps (recursive level step) + 1 adaptation",
                "parallelism": "replicas" if world > 1 else "single GPU",
                "l2": "flushed between timed steps (256 MiB write, untimed)",
                "coarse_step_at_start": start_counts["coarse_steps"],
                "blocks_per_level_start": start_counts["n_ids"],
                "blocks_per_level_end": end_counts["n_ids"],
                "leaf_updates_per_coarse_step_end": leaf_updates_end,
                "solver_mlups_excl_adapt": round(updates / t_solver / 1e6, 2),
                "window_mlups": [round(w, 1) for w in win],
                "median_window_mlups": round(float(sorted(win)[len(win) // 2]), 1) if win else None,
                "active_cell_mlups": round(active_updates / t_total / 1e6, 2),
                "section51_mean": {
                    "mlups": round(float(np.mean(inst)), 1) if inst else None,
                    "samples": len(inst),
                    "coarse_step_at_start": section51_start,
                    "note": "context, not the headline: the mean of the instantaneous MLUPS "
                            "of single coarse steps (CUDA events around each, solver only, "
                            "no L2 flush), as Section 5.1 averages its last 1024 samples; "
                            "measured after the timed and end-to-end steps, on the mesh of "
                            "that later time"},
                "mlups_count": "leaf-cell updates, sum_L 2^L (N_L - N_(L+1)/N_c) M (Section 5.1); "
                               "active_cell_mlups also counts the refined blocks advanced at the "
                               "coarse-fine interface",
                "adapt_share": round(1 - t_solver / t_total, 4),
                "capacity_errors": int(capacity_errors),
                "kernels_sampled": share,
                "adapt_phase_ms_per_adaptation": adapt_phases,
                "baseline": "paper A100 mean MLUPS 1753 (D3Q19 FP32 64^3, L_max 4): context",
                "uniform_bar": bar,
            },
            "roofline": roof,
            "e2e": {"value": round(e2e_updates / t_e2e / 1e6, 2), "unit": "MLUP/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": nbytes,
                    "note": "amr_step + amr_adapt + amr_fields(AMR_RHO_U) to pinned host "
                            "memory every step",
                    "h2d_reason": "no per-step input: a lid-driven cavity started from rest "
                                  "is defined by its configuration (amr_init builds the rest "
                                  "state on the device); each step's result (rho and u of "
                                  "every block, d2h_bytes_per_step) is read back to the host"},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
    sim.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_bar(args, AmrLBM, W, torch, dev, stream, order="lexicographic"):
    """Single-level periodic D3Q19 FP32 forest of 256^3 cells (2 x 1.27 GB of
    populations, far above L2): fused collide-stream only.  `order` numbers
    the root blocks lexicographically, along the Morton curve or by a seeded
    shuffle (block IDs then carry no spatial locality)."""
    cfg = W.config_uniform_bar(256)
    if order == "morton":
        cfg["root_ids"] = W.morton_root_ids(cfg)
    elif order == "shuffled":
        cfg["root_ids"] = W.shuffled_root_ids(cfg, 0)
    sim = AmrLBM(cfg, storage="f32", kernel_variant=args.variant)
    sim.step(3)
    sim.profile(1)
    sim.profile_read(reset=True)
    n = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sim.profile_read(reset=True)["collide_stream"]
    sim.close()
    peak, _ = measured_peaks()
    ups = 256 ** 3
    kernel_gbs = prof["bytes"] / (prof["ms"] / 1e3) / 1e9
    return {"cells": ups, "variant": args.variant, "root_order": order,
            "mlups": round(ups * n / (e0.elapsed_time(e1) / 1e3) / 1e6, 1),
            "kernel_gbs": round(kernel_gbs, 1), "frac": round(kernel_gbs / peak, 4)}


# ------------------------------------------------------- cylinder workload
def run_cylinder(args):
    """Channel past a square prism, D3Q27 BGK, FP32 arithmetic with FP64 /
    FP32 / BF16 / FP16 storage on one static mesh (distance refinement with
    freezing, vorticity refinement off so every storage sees the same mesh).
    Reports MLUPS per storage, relative L2 of rho and u per level against the
    FP64 run, and the drag coefficient from the momentum-exchange force."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AMR_RHO_U, AmrLBM
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    nx = args.cyl_nx
    scale = nx / 256
    cfg = W.channel_cylinder(q=27, nx=nx, ny=int(64 * scale), nz=int(64 * scale),
                             side=8 * scale, cx=64 * scale, cy=32 * scale,
                             max_levels=args.cyl_levels, crit_start=100, crit_inc=1,
                             max_blocks=args.cyl_cap)
    u0, side = 0.05, 8 * scale
    area = (side / nx) * (cfg["nz"] / nx)           # D * H in physical units (length_x = 1)
    results, refs = {}, {}
    runs = [(st, it) for it in args.cyl_interp.split(",") for st in args.cyl_storages.split(",")]
    for storage, interp in runs:
        cfg["interp"] = interp
        sim = AmrLBM(cfg, storage=storage, kernel_variant=args.variant)
        for _ in range(args.cyl_levels):            # static distance-refined mesh
            sim.adapt()
        counts = sim.counts()
        ups = sim.updates_per_coarse_step()
        sim.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        forces = []
        n_done = 2
        t_ms = 0.0
        while n_done < args.cyl_steps:
            chunk = min(16, args.cyl_steps - n_done)
            e0.record(stream)
            sim.step(chunk)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            n_done += chunk
            forces.append(sim.force()[0])
        rho_u = sim.fields_device(AMR_RHO_U, torch.float64).reshape(sim.cap, sim.m, 4)
        lev = torch.from_numpy(sim.blocks()["level"]).to(dev)
        tail = forces[int(0.8 * len(forces)):] or forces[-1:]
        cd = [2.0 * f / (u0 * u0 * area) for f in tail]
        entry = {"mlups": round(ups * (n_done - 2) / (t_ms / 1e3) / 1e6, 1),
                 "blocks_per_level": counts["n_ids"], "leaf_updates_per_coarse_step": ups,
                 "coarse_steps": n_done, "C_D_last20pct_mean": float(np.mean(cd)),
                 "interp": interp,
                 "bytes_per_update": 2 * 27 * {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage]}
        ref = refs.get(interp)
        if ref is None:
            refs[interp] = rho_u
        else:
            per_level = {}
            for L in range(cfg["max_levels"]):
                sel = lev == L
                if not bool(sel.any()):
                    continue
                a, b = rho_u[sel], ref[sel]
                per_level[L] = {
                    "rho": float(torch.linalg.norm(a[..., 0] - b[..., 0]) / torch.linalg.norm(b[..., 0])),
                    "u": float(torch.linalg.norm(a[..., 1:] - b[..., 1:]) / torch.linalg.norm(b[..., 1:]))}
            entry["rel_l2_vs_first"] = per_level
        results[storage if interp == "linear" else storage + "_" + interp] = entry
        del rho_u
        sim.close()
        torch.cuda.empty_cache()
    return {"workload": "channel past a square prism, D3Q27, %dx%dx%d root cells, side %g, "
                        "Re 100, L_max %d, static distance refinement (0.15/2^L, frozen)" %
                        (nx, cfg["ny"], cfg["nz"], side, cfg["max_levels"]),
            "reference_storage": args.cyl_storages.split(",")[0] + " (per interpolation)",
            "results": results}


# --------------------------------------------- FP32 against FP64 (cavity)
def centreline_profiles(sim, n_pts=256):
    """u_x along the vertical centreline (x = y = half width, z from bottom to
    lid) and u_z along the horizontal centreline (y = z = half width, x from
    wall to wall) of a 3D cavity, each sampled at n_pts evenly spaced points
    from the leaf cell that contains the point (after the level
    synchronisation)."""
    import numpy as np
    rho, u = sim.rho_u()
    blk = sim.blocks()
    X = sim.coords()
    lev, st = blk["level"], blk["status"]
    n = sim.cfg["nx"]
    leaves = np.nonzero(st == 1)[0]
    w = 4.0 / 2.0 ** lev[leaves]
    lo = X[leaves]
    hi = lo + w[:, None]
    s = (np.arange(n_pts) + 0.5) * n / n_pts
    h = n / 2.0

    def sample(pts, comp):
        out = np.empty(len(pts))
        for i, pnt in enumerate(pts):
            k = np.nonzero(np.all((lo <= pnt) & (pnt < hi), axis=1))[0][0]
            b = leaves[k]
            cell = np.floor((pnt - X[b]) / (w[k] / 4.0)).astype(int)
            out[i] = u[b, cell[0] + 4 * cell[1] + 16 * cell[2], comp]
        return out

    vert = np.stack([np.full(n_pts, h), np.full(n_pts, h), s], 1)
    horz = np.stack([s, np.full(n_pts, h), np.full(n_pts, h)], 1)
    return sample(vert, 0), sample(horz, 2)


def run_compare(args):
    """The 3D cavity of the headline (64^3 root cells, D3Q19, Re 1000, L_max 4,
    the vorticity criterion every 50 coarse steps) run from rest in FP64 and in
    FP32 storage and arithmetic for --cmp-steps coarse steps; reports MLUPS of
    each and the relative L2 difference of the centreline velocity profiles
    (the two runs adapt on their own, so their meshes may differ)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out, prof = {}, {}
    for storage in ("f64", "f32"):
        cfg = W.config_c1(n=args.n, max_blocks=(args.n // 4) ** 3 * args.cap_factor)
        sim = AmrLBM(cfg, storage=storage)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        updates, ms, cap_err = 0.0, 0.0, 0
        for _ in range(args.cmp_steps // PERIOD):
            updates += PERIOD * sim.updates_per_coarse_step()
            e0.record(stream)
            sim.step(PERIOD)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            rc, _ = sim.adapt()
            cap_err += rc != 0
        prof[storage] = centreline_profiles(sim)
        out[storage] = {"mlups_excl_adapt": round(updates / (ms / 1e3) / 1e6, 1),
                        "blocks_per_level": sim.counts()["n_ids"], "capacity_errors": cap_err}
        sim.close()
        torch.cuda.empty_cache()
    a, b = prof["f32"], prof["f64"]
    return {"workload": "3D lid-driven cavity D3Q19, %d^3 root cells, Re 1000, L_max 4, "
                        "criterion every 50 coarse steps, from rest" % args.n,
            "coarse_steps": (args.cmp_steps // PERIOD) * PERIOD, "runs": out,
            "rel_l2_f32_vs_f64": {
                "u_x_vertical_centreline": float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])),
                "u_z_horizontal_centreline": float(np.linalg.norm(a[1] - b[1]) / np.linalg.norm(b[1]))},
            "profiles_f64": {"u_x_vertical": [round(v, 6) for v in b[0][::8]],
                             "u_z_horizontal": [round(v, 6) for v in b[1][::8]]}}


# ------------------------------------------------ Strouhal number (quasi-2D)
def fit_sinusoid(t, y):
    """Frequency, amplitude and mean of the sinusoid that fits y(t) best in
    least squares: the FFT peak, refined by a scan of the residual of the
    linear fit of (sin, cos, 1) at frequencies around it."""
    import numpy as np
    t = np.asarray(t, float)
    y = np.asarray(y, float)
    dt = t[1] - t[0]
    spec = np.abs(np.fft.rfft(y - y.mean()))
    freqs = np.fft.rfftfreq(len(y), dt)
    k = int(np.argmax(spec[1:]) + 1)
    best = None
    for f in np.linspace(freqs[max(k - 1, 1)], freqs[min(k + 1, len(freqs) - 1)], 801):
        A = np.stack([np.sin(2 * np.pi * f * t), np.cos(2 * np.pi * f * t), np.ones_like(t)], 1)
        coef, res, _, _ = np.linalg.lstsq(A, y, rcond=None)
        r = float(np.sum((A @ coef - y) ** 2))
        if best is None or r < best[0]:
            best = (r, f, float(np.hypot(coef[0], coef[1])), float(coef[2]))
    return best[1], best[2], best[3]


def run_strouhal(args):
    """Quasi-2D flow past a square prism (the paper's FPSC case, Section 5.3):
    D3Q19, 256 x 64 root cells, one block span with periodic z faces, prism
    of side 8 one cell above the channel centre (to break the symmetry), Re
    100, inlet 0.05, static distance refinement around the prism and the
    outlet.  The lift coefficient is sampled every 16 coarse steps; after
    --st-spinup coarse steps a sinusoid is fitted to it: St = f D / U."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM
    torch.cuda.set_device(0)
    side, u0, nx = 8.0, 0.05, 256
    out = {}
    for interp in args.st_interp.split(","):
        if args.st_dim == 2:
            # the paper's 2D case: a 32 D x 32 D domain (256^2 root cells, D = 8),
            # the prism 10 D downstream, one cell above the centre line
            cfg = W.channel_cylinder(dim=2, nx=nx, ny=nx, side=side, cx=80, cy=129,
                                     max_levels=args.st_levels, crit_start=100, crit_inc=1,
                                     max_blocks=4096 * 40)
        else:
            cfg = W.channel_cylinder(q=19, nx=nx, ny=64, nz=4, side=side, cx=64, cy=33,
                                     max_levels=args.st_levels, crit_start=100, crit_inc=1,
                                     max_blocks=1024 * 40, span_periodic=True)
        cfg["interp"] = interp
        sim = AmrLBM(cfg, storage="f64" if args.st_dim == 2 else "f32")
        for _ in range(args.st_levels):
            sim.adapt()
        area = (side / nx) * ((cfg["nz"] / nx) if args.st_dim == 3 else 1.0)
        t, cl, cd = [], [], []
        n = 0
        t0 = time.perf_counter()
        while n < args.st_steps:
            sim.step(16)
            n += 16
            if n >= args.st_spinup:
                fx, fy, _ = sim.force()
                t.append(n)
                cl.append(2.0 * fy / (u0 * u0 * area))
                cd.append(2.0 * fx / (u0 * u0 * area))
        wall = time.perf_counter() - t0
        f, amp, mean = fit_sinusoid(t, cl)
        out[interp] = {"St": round(f * side / u0, 4), "C_L_amplitude": round(amp, 4),
                       "C_L_mean": round(mean, 4), "C_D_mean": round(float(np.mean(cd)), 4),
                       "periods_fitted": round(f * (t[-1] - t[0]), 1),
                       "blocks_per_level": sim.counts()["n_ids"],
                       "wall_s": round(wall, 1)}
        sim.close()
    if args.st_dim == 2:
        name = ("2D flow past a square cylinder (Section 5.3), D2Q9 FP64, 256^2 root cells "
                "(32 D x 32 D), D = 8, prism 10 D downstream, Re 100, L_max %d" % args.st_levels)
    else:
        name = ("quasi-2D channel past a square prism, D3Q19, 256x64 root cells, span one block "
                "(periodic), side 8, Re 100, L_max %d" % args.st_levels)
    return {"workload": name,
            "coarse_steps": args.st_steps, "spinup": args.st_spinup, "results": out}


# --------------------------------------- the paper's MLUPS table on this GPU
PAPER_A100_TABLE = {  # mean MLUPS on an A100 (FP32, FP64), lid-driven cavities, L_max 4
    "D2Q9 128^2": (495.0, 452.0), "D3Q19 64^3": (1753.0, 1219.0),
    "D3Q27 64^3": (1089.0, 786.0)}


def run_table(args):
    """The paper's MLUPS table for lid-driven cavities (D2Q9 at 128^2 root
    cells, D3Q19 and D3Q27 at 64^3, L_max 4, Re 1000, the vorticity criterion
    every 50 coarse steps) in FP32 and FP64, with the benchmark's protocol:
    --warmup periods of 50 coarse steps + adaptation, then --steps timed
    periods; the paper's A100 means are given as context."""
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rows = []
    for name, dim, q, n in (("D2Q9 128^2", 2, 9, 128), ("D3Q19 64^3", 3, 19, 64),
                            ("D3Q27 64^3", 3, 27, 64)):
        for k, storage in enumerate(("f32", "f64")):
            roots = (n // 4) ** dim
            cfg = W.cavity(dim=dim, q=q, n=n, re=1000.0, max_levels=4, max_blocks=roots * 128)
            sim = AmrLBM(cfg, storage=storage)
            for _ in range(args.warmup):
                sim.step(PERIOD)
                sim.adapt()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            upd, t_all, t_solve = 0.0, 0.0, 0.0
            for _ in range(args.steps):
                upd += PERIOD * sim.updates_per_coarse_step()
                e0.record(stream)
                sim.step(PERIOD)
                e1.record(stream)
                sim.adapt()
                e2.record(stream)
                torch.cuda.synchronize()
                t_all += e0.elapsed_time(e2) / 1e3
                t_solve += e0.elapsed_time(e1) / 1e3
            rows.append({"case": name, "storage": storage,
                         "mlups": round(upd / t_all / 1e6, 1),
                         "mlups_excl_adapt": round(upd / t_solve / 1e6, 1),
                         "blocks_per_level": sim.counts()["n_ids"],
                         "paper_a100_mlups": PAPER_A100_TABLE[name][k],
                         "ratio_to_a100": round(upd / t_all / 1e6 / PAPER_A100_TABLE[name][k], 1)})
            sim.close()
            torch.cuda.empty_cache()
    return {"workload": "lid-driven cavities, Re 1000, L_max 4, criterion every 50 coarse steps",
            "warmup_periods": args.warmup, "timed_periods": args.steps, "rows": rows}


# ------------------------------------------- cell vs. block arrangement (E6)
# block / cell time ratios of the paper's single-level comparison (A100), by
# arrangement, for D2Q9 2048^2, D3Q19 192^3, D3Q27 192^3: context only
PAPER_E6_RATIO = {"calculated": (1.73, 1.39, 1.47), "retrieved": (1.58, 1.25, 1.34),
                  "morton": (1.58, 1.12, 1.15), "shuffled": (0.39, 0.44, 0.33)}


def run_e6(args):
    """Cell- against block-based arrangement on one level (the paper's
    comparison, Section 5): periodic D2Q9 2048^2, D3Q19 192^3 and D3Q27 192^3
    grids, FP32, from rest.  Cell-based: one element per cell with x-fastest
    IDs and computed neighbours ('calculated'), the same IDs with neighbours
    from a table ('retrieved'), Morton IDs, or shuffled IDs (table).
    Block-based: the single-level block forest with its root blocks numbered
    lexicographically (it always reads neighbours from its table: it serves
    both structured rows), along the Morton curve, or shuffled.  Time per step
    from CUDA events over --e6-steps launches after 5 warm-up steps; the
    working sets exceed L2."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM, Cells
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()
    nsteps = args.e6_steps
    rows = []

    def timed(step_fn):
        step_fn(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step_fn(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / nsteps

    for ci, (name, dim, q, shape) in enumerate((("D2Q9 2048^2", 2, 9, [2048, 2048]),
                                                ("D3Q19 192^3", 3, 19, [192] * 3),
                                                ("D3Q27 192^3", 3, 27, [192] * 3))):
        n = int(np.prod(shape))
        nu0 = 0.01
        cell_t = {}
        for arr in W.CELL_ARRANGEMENTS:
            sim = Cells(dim, q, shape, nu0, W.cell_ids(shape, arr, seed=0))
            sim.set_rest()
            cell_t[arr] = timed(sim.step)
            del sim
            torch.cuda.empty_cache()
        block_t = {}
        for order in ("lexicographic", "morton", "shuffled"):
            cfg = W.periodic_box(dim=dim, q=q, n=shape[0], nu0=nu0, max_levels=1,
                                 max_blocks=n // 4 ** dim)
            if order == "morton":
                cfg["root_ids"] = W.morton_root_ids(cfg)
            elif order == "shuffled":
                cfg["root_ids"] = W.shuffled_root_ids(cfg, 0)
            sim = AmrLBM(cfg, storage="f32")
            block_t[order] = timed(sim.step)
            sim.close()
            torch.cuda.empty_cache()
        block_of = {"calculated": "lexicographic", "retrieved": "lexicographic",
                    "morton": "morton", "shuffled": "shuffled"}
        alg = 2 * q * 4 * n
        for arr in W.CELL_ARRANGEMENTS:
            tc, tb = cell_t[arr], block_t[block_of[arr]]
            rows.append({"case": name, "arrangement": arr,
                         "cell_us": round(tc * 1e6, 1), "block_us": round(tb * 1e6, 1),
                         "ratio_block_over_cell": round(tb / tc, 3),
                         "paper_ratio_a100": PAPER_E6_RATIO[arr][ci],
                         "cell_frac": round(alg / tc / 1e9 / peak, 4),
                         "block_frac": round(alg / tb / 1e9 / peak, 4),
                         "block_numbering": block_of[arr]})
    return {"workload": "cell- vs block-based arrangement, one level, periodic, FP32, from rest",
            "steps": nsteps, "peak_gbs": peak, "peak_source": peak_kind,
            "bytes_per_update": "2 Q 4 (neighbour tables not counted)", "rows": rows}


# ------------------------------------------------ adaptation cost sweep (E4)
def run_adapt_sweep(args):
    """Adaptation time against the number of inserted blocks (the paper's
    insertion sweep): a periodic 3D D3Q19 FP32 forest of 128^3 root cells
    (32,768 root blocks); seeded refine marks on a fraction of the roots,
    adapt, then coarsen them all back; device time per phase from the profile
    events and host wall time of the call."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM
    torch.cuda.set_device(0)
    n = 128
    roots = (n // 4) ** 3
    cfg = W.periodic_box(dim=3, q=19, n=n, nu0=0.01, max_levels=2, max_blocks=roots * 9)
    rows = []
    warm = AmrLBM(W.periodic_box(dim=3, q=19, n=16, nu0=0.01, max_levels=2, max_blocks=64 * 9),
                  storage="f32")
    warm.adapt(torch.ones(warm.cap, dtype=torch.int8, device="cuda"))
    warm.close()
    for frac in (0.003, 0.03, 0.1, 0.3, 1.0):
        sim = AmrLBM(cfg, storage="f32")
        sim.profile(1)
        m = (W.rng(7).random(sim.cap) < frac).astype(np.int8)
        m[roots:] = 0
        out = {}
        for kind, marks in (("refine", m), ("coarsen", -m)):
            sim.profile_read(reset=True)
            rc, st = sim.adapt(torch.from_numpy(marks).cuda())
            prof = sim.profile_read(reset=True)
            phases = {k[len("adapt_"):]: round(v["ms"], 4) for k, v in prof.items()
                      if k.startswith("adapt_")}
            out[kind] = {"blocks_changed": int(st["n_refined" if kind == "refine" else
                                                  "n_coarsened"]) * 8,
                         "host_ms": round(st["ms_total"], 3),
                         "device_ms": round(sum(phases.values()), 3), "phases_ms": phases}
        rows.append(out)
        sim.close()
        torch.cuda.empty_cache()
    return {"workload": "periodic 3D D3Q19 FP32 forest, 128^3 root cells (32,768 root blocks), "
                        "seeded refinement of a fraction of the roots, then coarsening back",
            "rows": rows}


# -------------------------------------------------------- batched workload
def run_batched(args):
    """64 independent 3D cavities (D3Q19 FP32) with seeded uneven sizes (32^3 to
    64^3 root cells), depths (0 to 3 extra levels) and Reynolds numbers
    (uniform in [100, 3200]).  Members that become BGK-unstable (tau_0 close
    to 1/2 on the coarsest grids) within a screening run as long as the
    measurement are left out before anything is timed, and listed.  The autotuner times the graph form (one launch per
    level operation, CUDA graph), the persistent form (one launch per call,
    M_L x threads) and the member-graph form (the members' own coarse steps
    as branches of one graph); the best of each form is timed over the same
    periods with the per-member adaptations between them, and compared with
    the same members advanced one by one.  Per-member relative L2 of rho and u after
    one period, batched against the same members advanced one by one from the
    same state (plain FP32 runs), on every 8th member."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AMR_RHO_U, AmrBatch, AmrLBM
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n = args.batch_n
    cfgs = W.batched_cavities(n, seed=0)

    def stable(m):
        try:
            return bool(np.all(np.isfinite(m.mass())))
        except Exception:
            return False

    # screening: every member for as many coarse steps as the measurement
    # below takes (warm-up, autotuning, three timed forms, sequential, L2),
    # untimed; members that become BGK-unstable are left out
    screen_periods = args.warmup + 2 + 4 * args.steps + 2
    members = [AmrLBM(cfg, storage="f32") for cfg in cfgs]
    batch = AmrBatch(members)
    for _ in range(screen_periods):
        batch.step(PERIOD)
        for m in members:
            m.adapt()
        batch.refresh()
    keep = [i for i, m in enumerate(members) if stable(m)]
    batch.close()
    for m in members:
        m.close()
    torch.cuda.empty_cache()
    excluded = [{"member": i, "n": cfgs[i]["nx"],
                 "re": round(0.05 * cfgs[i]["nx"] / cfgs[i]["nu0"], 1),
                 "tau0": round(3.0 * cfgs[i]["nu0"] + 0.5, 5)} for i in range(n) if i not in keep]
    members = [AmrLBM(cfgs[i], storage="f32") for i in keep]
    batch = AmrBatch(members)
    cap_err = 0
    for _ in range(args.warmup):
        batch.step(PERIOD)
        for m in members:
            cap_err += m.adapt()[0] != 0
        batch.refresh()
    # both forms tuned on the refined meshes; it advances the members
    chosen, times = batch.autotune(trial_steps=2)
    for m in members:
        cap_err += m.adapt()[0] != 0
    batch.refresh()
    torch.cuda.synchronize()

    def ups():
        return sum(m.updates_per_coarse_step() for m in members)

    best = {}
    for (form, t, ml), ms in times.items():
        if form not in best or ms < best[form][1]:
            best[form] = ((form, t, ml), ms)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timed = {}
    for form in ("graph", "persistent", "members"):
        (f, t, ml), _ = best[form]
        batch.configure(f, t, ml)
        tb = ta = 0.0
        upd = 0
        l0 = batch.launches()
        for _ in range(args.steps):
            upd += PERIOD * ups()
            e0.record(stream)
            batch.step(PERIOD)
            e1.record(stream)
            batch.sync()
            tb += e0.elapsed_time(e1) / 1e3
            h0 = time.perf_counter()
            for m in members:
                cap_err += m.adapt()[0] != 0
            batch.refresh()
            torch.cuda.synchronize()
            ta += time.perf_counter() - h0
        timed[form] = {"threads_per_cta": t, "blocks_per_tile": ml,
                       "mlups_step": round(upd / tb / 1e6, 1),
                       "mlups_with_adapt": round(upd / (tb + ta) / 1e6, 1),
                       "launches_per_period": (batch.launches() - l0) / args.steps}
    for m in members:                          # build each member's own graphs (untimed)
        m.step(1)
    for m in members:
        m.step(1)                              # back to the batch's buffer parity
    torch.cuda.synchronize()
    t_s = 0.0
    upd_s = 0
    l1 = sum(m.launches() for m in members)
    for _ in range(args.steps):
        upd_s += PERIOD * ups()
        e0.record(stream)
        for m in members:
            m.step(PERIOD)
        e1.record(stream)
        torch.cuda.synchronize()
        t_s += e0.elapsed_time(e1) / 1e3
    launches_s = sum(m.launches() for m in members) - l1
    seq = round(upd_s / t_s / 1e6, 1)
    # per-member L2, batched (chosen form) against one by one from one state
    batch.configure(chosen["form"], chosen["threads"], chosen["tile_blocks"])
    sample = list(range(0, len(members), 8))
    images = {i: members[i].checkpoint() for i in sample}
    batch.step(PERIOD)
    batch.sync()
    got = {i: members[i].fields_device(AMR_RHO_U, torch.float64) for i in sample}
    l2 = []
    for i in sample:
        members[i].restore(images[i])
        members[i].step(PERIOD)
        want = members[i].fields_device(AMR_RHO_U, torch.float64)
        l2.append(float(torch.linalg.norm(got[i] - want) / torch.linalg.norm(want)))
        del want
    unstable_end = sum(0 if stable(m) else 1 for m in members)
    blocks = [sum(m.counts()["n_ids"]) for m in members]
    win = max(timed, key=lambda k: timed[k]["mlups_step"])
    out = {"workload": "%d 3D lid-driven cavities D3Q19 FP32, root 32^3..64^3, 0..3 extra "
                       "levels, Re uniform in [100, 3200] (seed 0), lid 0.05" % n,
           "members_timed": len(members),
           "excluded_unstable_in_screening": excluded,
           "screening_coarse_steps": screen_periods * PERIOD,
           "autotuned": chosen,
           "autotune_ms_per_coarse_step": {"%s/%d threads/M_L %d" % k: round(v, 3)
                                           for k, v in sorted(times.items())},
           "blocks_min_max_total": [min(blocks), max(blocks), sum(blocks)],
           "graph_form": timed["graph"], "persistent_form": timed["persistent"],
           "member_graph_form": timed["members"],
           "sequential_mlups_step": seq,
           "launches_per_period_sequential": launches_s / args.steps,
           "faster_form": win,
           "persistent_over_graph": round(timed["persistent"]["mlups_step"] /
                                          timed["graph"]["mlups_step"], 3),
           "members_over_graph": round(timed["members"]["mlups_step"] /
                                       timed["graph"]["mlups_step"], 3),
           "speedup_step_over_sequential": round(timed[win]["mlups_step"] / seq, 3),
           "per_member_rel_l2_rho_u_vs_individual_fp32":
               {"members": sample, "max": max(l2), "median": float(np.median(l2))},
           "capacity_errors": int(cap_err), "unstable_at_end": unstable_end,
           "periods_timed": args.steps, "coarse_steps_per_period": PERIOD}
    batch.close()
    for m in members:
        m.close()
    return out


# ---------------------------------------------------------- learned workload
def run_learned(args):
    """Learned refinement proposal on the channel past a square prism (D3Q27,
    FP32, distance + vorticity criterion).  Training pairs: block summaries at
    t and the plain criterion's refine flag at t + 20 coarse steps, from seeded
    runs (seed s sets Re = 100 (0.8 + 0.05 s)); seeds 1-6 train, 7-8 test.
    Evaluation from one spun-up state: the plain criterion every 50, 100 and
    200 coarse steps, and proposal + criterion every 200.  Measures of late
    refinement (see evaluate): the time-averaged under-refined leaf fraction,
    and the missed rate at t + 20 on a shadow copy, both over leaves the
    adaptation could refine.  With --learn-fp64-ref: the relative L2 of u on
    two wake lines at the end of each mode against an FP64 run of the plain
    criterion every 50 steps from the same spun-up state."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AMR_BLOCKS, AMR_NBR, AMR_RHO_U, AmrLBM, Mlp
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    nx = args.cyl_nx
    sc = nx / 256

    def cfg_for(seed):
        return W.channel_cylinder(q=27, nx=nx, ny=int(64 * sc), nz=int(64 * sc), side=8 * sc,
                                  cx=64 * sc, cy=32 * sc, re=100.0 * (0.8 + 0.05 * seed),
                                  max_levels=args.cyl_levels, max_blocks=args.cyl_cap,
                                  crit_start=args.learn_crit_start)

    cap_errors = {"spin": 0}

    def spun_up(seed, storage="f32"):
        sim = AmrLBM(cfg_for(seed), storage=storage)
        for _ in range(args.learn_spin):
            sim.step(50)
            cap_errors["spin"] += sim.adapt()[0] != 0
        return sim

    # ---- training pairs
    per_seed = args.learn_pairs // 8
    xs, ys, seeds = [], [], []
    for seed in range(1, 9):
        sim = spun_up(seed)
        px, py = [], []
        for _ in range(args.learn_windows):
            feats = sim.features()

            leaf = torch.from_numpy(sim.blocks()["status"] == 1).to(dev)
            sim.step(20)
            flag = sim.criterion_marks() > 0
            px.append(feats[leaf])
            py.append(flag[leaf].float())
            sim.step(30)
            sim.adapt()
        x = torch.cat(px)
        y = torch.cat(py)
        stride = max(1, x.shape[0] // per_seed)
        xs.append(x[::stride][:per_seed].contiguous())
        ys.append(y[::stride][:per_seed].contiguous())
        seeds.append(seed)
        sim.close()
        torch.cuda.empty_cache()
    xtr, ytr = torch.cat(xs[:6]).contiguous(), torch.cat(ys[:6]).contiguous()
    xte, yte = torch.cat(xs[6:]).contiguous(), torch.cat(ys[6:]).contiguous()
    pos = float(ytr.sum())
    pw = max(1.0, (ytr.numel() - pos) / max(pos, 1.0))
    net = Mlp(dev, seed=0)
    t0 = time.perf_counter()
    losses = [net.train_epoch(xtr, ytr, batch=1024, lr=2e-3, pos_weight=pw, seed=e)
              for e in range(args.learn_epochs)]
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pr = net.infer(xte) > args.learn_threshold
    tp = float((pr & (yte > 0.5)).sum())
    test = {"pairs": int(xte.shape[0]), "positives": int(yte.sum()),
            "recall": tp / max(1.0, float(yte.sum())),
            "precision": tp / max(1.0, float(pr.sum())),
            "accuracy": float((pr.float() == yte).float().mean())}

    # ---- evaluation from one spun-up state (deterministic: equal histories).
    # Two measures of refinement that came too late:
    # * under-refinement: every `sample_every` coarse steps the plain
    #   criterion is evaluated on the running mesh without adapting; the
    #   fraction of leaves it would refine that the mesh could refine (leaf
    #   below the finest level with every same-level neighbour present: the
    #   eligibility rule of the adaptation) is averaged over the run;
    # * missed at t + 20: a shadow copy skips each adaptation for 20 coarse
    #   steps; of the eligible leaves the plain criterion flags there, the
    #   fraction that the adaptation at t did not refine (windows whose
    #   adaptation hit the capacity are left out and counted).  The shadow
    #   then applies the same marks, so both meshes stay identical.
    lmax = args.cyl_levels
    every = args.learn_sample_every

    def eligible_flagged(sim):
        marks = sim.criterion_marks()
        blk = sim.fields_device(AMR_BLOCKS, torch.int32).reshape(4, sim.cap)
        nbr = sim.fields_device(AMR_NBR, torch.int32).reshape(sim.cap, -1)
        leaf = blk[1] == 1
        elig = leaf & (blk[0] < lmax - 1) & ~(nbr == -1).any(1)
        del nbr
        return (marks > 0) & elig, leaf

    def evaluate(mode, period, shadow_on):
        main = spun_up(9)
        shadow = spun_up(9) if shadow_on else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ups_sum, t_ms, adapts, cap_err = 0.0, 0.0, 0, 0
        flagged = missed = skipped = 0
        under = []
        steps = 0

        def timed(fn):
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return r, e0.elapsed_time(e1)

        while steps < args.learn_eval_steps:
            def adapt_main():
                if mode == "learned":
                    m = main.propose_marks(net.half, args.learn_threshold, True)
                else:
                    m = main.criterion_marks()
                return m, main.adapt(m)[0]
            (marks, rc), ms = timed(adapt_main)
            t_ms += ms
            cap_err += rc != 0
            adapts += 1
            ups = main.updates_per_coarse_step()
            done = 0
            while done < period:
                k = min(every, period - done)
                t_ms += timed(lambda: main.step(k))[1]
                done += k
                f, leaf = eligible_flagged(main)
                under.append(float(f.sum()) / max(1.0, float(leaf.sum())))
                if shadow is not None and done == 20:
                    shadow.step(20)
                    want, _ = eligible_flagged(shadow)
                    if rc == 0:
                        still = main.fields_device(AMR_BLOCKS, torch.int32).reshape(4, main.cap)[1] == 1
                        flagged += int(want.sum())
                        missed += int((want & still).sum())
                    else:
                        skipped += 1
                    shadow.adapt(marks)
                    shadow.step(period - 20)
            ups_sum += ups * period
            steps += period
        if ref_lines is not None:
            got = wake_lines(main)
            out_l2 = float(np.linalg.norm(got - ref_lines) / np.linalg.norm(ref_lines))
        out = {"period": period, "mlups_incl_adapt": round(ups_sum / (t_ms / 1e3) / 1e6, 1),
               "adaptations": adapts, "coarse_steps": steps,
               "under_refined_leaf_fraction": round(float(np.mean(under)), 5),
               "capacity_errors": cap_err, "blocks_end": main.counts()["n_ids"]}
        if ref_lines is not None:
            out["rel_l2_wake_lines_vs_fp64_plain_every_50"] = round(out_l2, 6)
        if shadow is not None:
            out["missed_at_t_plus_20"] = {"eligible_flagged": flagged, "missed": missed,
                                          "rate": round(missed / max(1, flagged), 4),
                                          "windows_left_out_capacity": skipped}
            shadow.close()
        main.close()
        torch.cuda.empty_cache()
        return out

    def wake_lines(sim):
        """u_x, u_y (lattice units of the root grid) on the wake centreline
        (y = prism centre, z = mid-span, from the prism's rear face to the
        outlet) and on the cross line two side lengths behind the prism, 128
        points each, from the leaf cell that holds each point."""
        side, cx, cy = 8 * sc, 64 * sc, 32 * sc
        ny, nz = int(64 * sc), int(64 * sc)
        s = (np.arange(128) + 0.5) / 128
        pts = np.concatenate([
            np.stack([cx + side / 2 + s * (nx - cx - side / 2), np.full(128, cy),
                      np.full(128, nz / 2)], 1),
            np.stack([np.full(128, cx + 2 * side), s * ny, np.full(128, nz / 2)], 1)])
        blk = sim.blocks()
        X = sim.coords()
        leaves = np.nonzero(blk["status"] == 1)[0]
        w = 4.0 / 2.0 ** blk["level"][leaves]
        lo, hi = X[leaves], X[leaves] + w[:, None]
        idx = np.empty(len(pts), np.int64)
        for i, pnt in enumerate(pts):
            k = np.nonzero(np.all((lo <= pnt) & (pnt < hi), axis=1))[0][0]
            b = leaves[k]
            cell = np.floor((pnt - X[b]) / (w[k] / 4.0)).astype(int)
            idx[i] = b * 64 + cell[0] + 4 * cell[1] + 16 * cell[2]
        ru = sim.fields_device(AMR_RHO_U, torch.float64).view(-1, 4)
        u = ru[torch.from_numpy(idx).to(dev)][:, 1:3].cpu().numpy()
        del ru
        return u.reshape(-1)

    ref_lines = None
    fp64_ref = None
    if args.learn_fp64_ref:
        ref = spun_up(9, "f64")
        for _ in range(args.learn_eval_steps // 50):
            ref.adapt()
            ref.step(50)
        ref_lines = wake_lines(ref)
        fp64_ref = {"blocks_end": ref.counts()["n_ids"]}
        ref.close()
        torch.cuda.empty_cache()

    shadow_on = not args.learn_no_shadow
    ev = {}
    for mode in args.learn_modes.split(","):
        if mode == "learned":
            ev["learned_every_200"] = evaluate("learned", 200, shadow_on)
        else:
            ev["plain_every_%d" % int(mode)] = evaluate("plain", int(mode), shadow_on)
    fr = [ev["plain_every_%d" % p]["under_refined_leaf_fraction"] for p in (50, 100, 200)
          if "plain_every_%d" % p in ev]
    return {"workload": "learned refinement proposal, channel past a square prism D3Q27 FP32, "
                        "%dx%dx%d root, L_max %d, criterion N_start %d" % (
                            nx, int(64 * sc), int(64 * sc), args.cyl_levels,
                            args.learn_crit_start),
            "pairs_train": int(xtr.shape[0]), "pairs_test": test["pairs"],
            "pos_weight": round(pw, 2), "epochs": args.learn_epochs,
            "loss_first_last": [round(losses[0], 4), round(losses[-1], 4)],
            "train_seconds": round(t_train, 3), "threshold": args.learn_threshold,
            "test": test, "capacity": args.cyl_cap,
            "capacity_errors_spin_up": int(cap_errors["spin"]),
            "under_refinement_monotone_in_period": bool(all(a <= b for a, b in zip(fr, fr[1:]))),
            "sample_every": every, "fp64_reference": fp64_ref, "evaluation": ev,
            "learned_speedup_over_plain_every_50": round(
                ev["learned_every_200"]["mlups_incl_adapt"] /
                ev["plain_every_50"]["mlups_incl_adapt"], 3)
            if "learned_every_200" in ev and "plain_every_50" in ev else None}


# ----------------------------------------------------------- reference arm
def run_oracle_timing(args):
    """The oracle's complete runs of the 2D cavity (C0: D2Q9 FP64, 64^2 root
    cells, 2000 coarse steps, criterion every 100) and of the benchmark
    cavity cut to 32^3 root cells (150 coarse steps, criterion every 50), on
    one core and on every core at once (one complete run per core), next to
    the GPU running the same inputs (FP64 for C0; FP32 and FP64 for the cut)
    through the library, adaptations included in every time."""
    import torch
    import workloads as W
    from paper_2308_08085_gb300 import AmrLBM
    info = cpu_info()
    n = max(1, info["nproc"] or 1)
    out = {"workload": "oracle timing", "cpu": info, "runs": {}}
    gpu_storages = {"c0": ["f64"], "c1cut": ["f32", "f64"]}
    for name, (mk, steps, every) in FULL_RUNS.items():
        row = {"coarse_steps": steps, "criterion_every": every}
        one = oracle_processes(1, 0, 1, 7200, run=name)
        if one:
            v, u, t = aggregate(one)
            row["oracle_one_core"] = {"mlups": round(v, 4), "seconds": round(t, 2),
                                      "updates": u, "mesh_end": one[0]["desc"]}
        alln = oracle_processes(n, 0, 1, 14400, run=name)
        if len(alln) == n:
            v, u, t = aggregate(alln)
            row["oracle_all_cores"] = {"mlups": round(v, 4), "seconds": round(t, 2),
                                       "processes": n}
        for st in gpu_storages[name]:
            cfg = mk(W)
            sim = AmrLBM(cfg, storage=st)
            torch.cuda.synchronize()
            upd = 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps // every):
                upd += every * sim.updates_per_coarse_step()
                sim.step(every)
                sim.adapt()
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            row["gpu_" + st] = {"mlups": round(upd / sec / 1e6, 1), "seconds": round(sec, 4)}
            sim.close()
        out["runs"][name] = row
    return out


def run_reference(args):
    """The oracle as it stands on the host cores (one process per core, each
    the bounded sample of OracleSample), `--warmup` + `--steps` steps of about
    120 s / (warmup + steps) each; a step's value is all processes' updates
    over the longest process time."""
    world, rank, local = dist_setup()
    if rank != 0:
        return None
    info = cpu_info()
    n = max(1, info["nproc"] or 1)
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    res = oracle_processes(n, per_step, args.warmup + args.steps,
                           per_step * (args.warmup + args.steps) * 20 + 600)
    if len(res) != n:
        return {"impl": "reference", "unavailable": "oracle worker processes failed"}
    value, upd, dt = aggregate(res, args.warmup)
    desc = res[0]["desc"]
    return {"impl": "reference", "metric": "MLUPS", "value": round(value, 4),
            "unit": "MLUP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / max(1, args.steps), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": CAVITY_WORKLOAD,
                       "sample": "each step a bounded sample of the workload: the same cavity "
                                 "cut to 32^3 root cells, run by the oracle in one process "
                                 "per host core"},
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUP/s", "cores": n,
                             "kind": "oracle", "sample": desc, "cpu_model": info["model"]},
            "e2e": {"value": round(value, 4), "unit": "MLUP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--cap-factor", type=int, default=128)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--paper-samples", type=int, default=1024,
                    help="single coarse steps timed for the Section 5.1 mean (0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-bar", action="store_true")
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cpu-run", default=None, choices=["c0", "c1cut"])
    ap.add_argument("--variant", type=int, default=0,
                    help="collide-stream kernel: 0 auto, 1 one-pass, 2/3 pipelined stages")
    ap.add_argument("--workload", default="cavity",
                    choices=["cavity", "cylinder", "batched", "learned", "compare", "strouhal",
                             "adapt", "table", "e6", "oracle"])
    ap.add_argument("--e6-steps", type=int, default=200)
    ap.add_argument("--st-steps", type=int, default=16000)
    ap.add_argument("--st-spinup", type=int, default=8000)
    ap.add_argument("--st-levels", type=int, default=3)
    ap.add_argument("--st-dim", type=int, default=3, choices=[2, 3],
                    help="2: the paper's 2D D2Q9 case; 3: quasi-2D D3Q19 span")
    ap.add_argument("--st-interp", default="linear,cubic")
    ap.add_argument("--cmp-steps", type=int, default=10000,
                    help="coarse steps of the FP32 / FP64 cavity comparison")
    ap.add_argument("--learn-pairs", type=int, default=200_000)
    ap.add_argument("--learn-spin", type=int, default=4)
    ap.add_argument("--learn-windows", type=int, default=4)
    ap.add_argument("--learn-epochs", type=int, default=12)
    ap.add_argument("--learn-threshold", type=float, default=0.5)
    ap.add_argument("--learn-eval-steps", type=int, default=800)
    ap.add_argument("--learn-sample-every", type=int, default=10)
    ap.add_argument("--learn-crit-start", type=int, default=-3)
    ap.add_argument("--learn-no-shadow", action="store_true")
    ap.add_argument("--learn-fp64-ref", action="store_true")
    ap.add_argument("--learn-modes", default="50,100,200,learned",
                    help="adaptation periods of the plain criterion, and 'learned'")
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--cyl-nx", type=int, default=256)
    ap.add_argument("--cyl-levels", type=int, default=5)
    ap.add_argument("--cyl-steps", type=int, default=400)
    ap.add_argument("--cyl-cap", type=int, default=4_000_000)
    ap.add_argument("--cyl-storages", default="f64,f32,bf16,f16")
    ap.add_argument("--cyl-interp", default="linear",
                    help="comma list of coarse-to-fine interpolations: linear, cubic")
    ap.add_argument("--bar-only", action="store_true",
                    help="only the single-level 256^3 D3Q19 FP32 forest (profiling)")
    ap.add_argument("--bar-order", default="lexicographic",
                    choices=["lexicographic", "morton", "shuffled"],
                    help="root-block numbering of the --bar-only forest")
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "cylinder":
        print(json.dumps(run_cylinder(args)))
        return
    if args.workload == "oracle":
        print(json.dumps(run_oracle_timing(args)))
        return
    if args.workload == "table":
        print(json.dumps(run_table(args)))
        return
    if args.workload == "e6":
        print(json.dumps(run_e6(args)))
        return
    if args.workload == "adapt":
        print(json.dumps(run_adapt_sweep(args)))
        return
    if args.workload == "strouhal":
        print(json.dumps(run_strouhal(args)))
        return
    if args.workload == "compare":
        print(json.dumps(run_compare(args)))
        return
    if args.workload == "batched":
        print(json.dumps(run_batched(args)))
        return
    if args.workload == "learned":
        print(json.dumps(run_learned(args)))
        return
    if args.bar_only:
        import torch
        import workloads as W
        from paper_2308_08085_gb300 import AmrLBM
        torch.cuda.set_device(0)
        print(json.dumps(run_bar(args, AmrLBM, W, torch, torch.device("cuda", 0),
                                 torch.cuda.current_stream(), args.bar_order)))
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out))
        return
    world, rank, local = dist_setup()
    out = run_ours(args)
    if rank == 0 and out is not None:
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = run_cpu_baseline(args.cpu_budget)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))


if __name__ == "__main__":
    main()
