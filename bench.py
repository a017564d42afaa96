#!/usr/bin/env python
"""Benchmark of the FP16-RCLL neighbour search + SPH density path on GB300.

One step = the whole hot path on one batch of synthetic input: binning
(bounds, cell hash, scan, scatter, per-cell sort, FP64 -> FP16/FP32
cell-relative conversion) and the search (count pass, row scan, fill pass with
the fused density), CSR in cell order.  Default workload: the 3D jittered
lattice of 1,000,000 particles (100^3, dx = 0.01, jitter +-0.1 dx, h = 1.3 dx,
kh = 2.6 dx).  Inputs are resident on the device when the timed region starts
and L2 is flushed (256 MiB write) between timed steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (the reference arm).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NNPS particles/s, FP16-RCLL vs FP64-CLL on 1 GB300 at 1M 3D; served p99 latency"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["3d_1m", "2d_10k", "3d_8m"], default="3d_1m")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-CLL, e2e and CPU-baseline legs")
    ap.add_argument("--side", type=int, default=100,
                    help="lattice side of the 3d_1m shape (100 = the 1,000,000-particle workload; "
                         "smaller sides are for profiler captures)")
    args = ap.parse_args()
    global SIDE
    SIDE = args.side
    return args


SIDE = 100


def workload(name):
    from paper_2401_08586_gb300 import workloads as W
    if name == "3d_1m":
        ps = W.c2_3d_1m(side=SIDE)
        desc = ("3d_1m_jittered_lattice: %d^3 lattice, dx=0.01, jitter U(+-0.1dx), "
                "h=1.3dx, kh=2.6dx, cell=kh, seed 2" % SIDE)
    elif name == "2d_10k":
        ps = W.c1_2d_10k()
        desc = "2d_10k_jittered_lattice: 100^2, dx=0.01, jitter U(+-0.1dx), h=1.2dx, kh=2h, seed 1"
    else:
        ps = W.c3_3d_dambreak()
        desc = ("3d_8m_dambreak: 200^3 lattice dx=1/200 in z<1 of a 1x1x2 box, 5% spray in z in (1,2], "
                "jitter U(+-0.2dx), h=1.5dx, kh=3dx, seed 3")
    return ps, desc


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("nnps_tile.cu", "nnps_common.cuh", "sph_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2401_08586_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name, kernel_tag):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload_name][kernel_tag]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.tmp, stderr=subprocess.DEVNULL)
            # the timed region starts only once the sampler is producing rows
            t_end = time.time() + 10.0
            while time.time() < t_end and os.path.getsize(self.tmp.name) == 0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        try:
            rows = [l.split(",") for l in open(self.tmp.name).read().strip().splitlines() if l.strip()]
            os.unlink(self.tmp.name)
        except Exception:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """FP64 CPU oracle (cell link-list + density) on the host cores."""
    if rank != 0:
        return 0
    import oracle
    ps, desc = workload(args.workload)
    threads = os.cpu_count() or 1
    oracle.build.build()

    def step():
        rp, col = oracle.cll(ps.xyz, ps.kh, threads=threads)
        oracle.density(ps.xyz, ps.h, rp, col, threads=threads)

    for _ in range(args.warmup):
        step()
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        t.append(time.perf_counter() - t0)
    total = sum(t)
    value = ps.n * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n_particles": ps.n},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": threads, "kind": "oracle",
                         "sample": "full workload per step (FP64 cell link-list + density, OpenMP rows)"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(ps, budget_s=12.0):
    """The oracle as it stands on all host cores, repeated for ~budget_s; and
    one single-threaded pass (the paper's CPU reference is one core)."""
    import oracle
    oracle.build.build()
    threads = os.cpu_count() or 1
    reps, t_total = 0, 0.0
    while t_total < budget_s and reps < 50:
        t0 = time.perf_counter()
        rp, col = oracle.cll(ps.xyz, ps.kh, threads=threads)
        oracle.density(ps.xyz, ps.h, rp, col, threads=threads)
        t_total += time.perf_counter() - t0
        reps += 1
    t0 = time.perf_counter()
    rp, col = oracle.cll(ps.xyz, ps.kh, threads=1)
    oracle.density(ps.xyz, ps.h, rp, col, threads=1)
    t1 = time.perf_counter() - t0
    return {"value": ps.n * reps / t_total, "unit": "particles/s", "cores": threads, "kind": "oracle",
            "sample": "%d full passes of the workload (%d particles each, FP64 cell link-list + density)"
                      % (reps, ps.n),
            "single_thread_value": ps.n / t1}


# ----------------------------------------------------------------- our arm

def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2401_08586_gb300 import sph

    sph.load(build_if_missing=True)
    ps, desc = workload(args.workload)
    n = ps.n
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    xyz = torch.from_numpy(ps.xyz).to(dev)
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)

    # capacity discovery (not timed)
    grid = sph.sph_bin_cells(params, xyz, n, sptr, None)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = sph.sph_nnps_query(grid, row_ptr, None, 0, True, None, sptr)
    cap = int(nnz * 1.02) + 1024
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(g):
        g = sph.sph_bin_cells(params, xyz, n, sptr, g)
        sph.sph_nnps_query(g, row_ptr, col, cap, False, rho, sptr)
        return g

    for _ in range(args.warmup):
        flush.fill_(1.0)
        grid = step(grid)
    torch.cuda.synchronize()
    sph.sph_grid_check(grid, sptr)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # timed region: CUDA events around the search kernel only (the roofline's
    # launch duration); every other launch runs without event overhead
    sph.sph_profile_reset()
    sph.sph_profile_select("fused,fill")
    launches0 = sph.sph_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            grid = step(grid)
            evs[k][1].record(stream)
        barrier()
        t1 = time.perf_counter()
    launches = sph.sph_launch_count() - launches0
    sph.sph_profile_enable(False)
    sph.sph_grid_check(grid, sptr)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([dev_total_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_total_s = float(t.item())
    value = world * n * args.steps / dev_total_s
    timed = {}
    for tag in ("fused", "fill"):
        ms, c = sph.sph_profile_read(tag)
        if c:
            timed[tag] = {"ms_total": ms, "launches": c}
    # phase breakdown (untimed): a few more steps with events around every launch
    sph.sph_profile_reset()
    sph.sph_profile_enable(True)
    nprof = min(args.steps, 10)
    for k in range(nprof):
        flush.fill_(float(k))
        grid = step(grid)
    torch.cuda.synchronize()
    sph.sph_profile_enable(False)
    sph.sph_grid_check(grid, sptr)  # reads back the last query's band counters
    phase = {}
    for tag in ("bounds", "hash", "scan", "scatter", "sort", "convert", "count", "fill", "fused"):
        ms, c = sph.sph_profile_read(tag)
        if c:
            phase[tag] = {"ms_total": ms, "launches": c}
    nnz = int(row_ptr[n].item())
    info = sph.sph_grid_info_get(grid)

    # roofline of the dominant kernel (the search: FP16 tests + FP32
    # re-decision + fused density + CSR write), algorithmic bytes per launch:
    # rel16 8 + rel32 16 + row_ptr 8 + rho 4 per particle, 4 per neighbour
    dom = "fused" if "fused" in timed else "fill"
    dom_ms = timed[dom]["ms_total"] / timed[dom]["launches"]
    alg_dom = n * (8 + 16 + 8 + 4) + 4 * nnz
    peak, peak_src = measured_peaks()
    achieved = alg_dom / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_nnps_tile" if dom == "fused" else "k_nnps<fill>",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src, "launch_ms": dom_ms, "algorithmic_bytes_per_launch": alg_dom,
                "traffic": ncu_traffic(args.workload, dom)}
    # whole path: binning 56 B/particle, search + fused density 36 B/particle + 4 B/neighbour
    alg_step = n * (56 + 36) + 4 * nnz
    step_ms_mean = 1e3 * dev_total_s / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms_mean, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": desc, "n_particles": n, "dim": ps.dim, "order": "cell",
                   "density": "fused, fp32 accumulation", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "roofline": roofline,
        "nnz": nnz, "neighbours_per_particle": nnz / n,
        "step_hbm_frac": alg_step / (step_ms_mean * 1e-3) / 1e9 / peak,
        "step_algorithmic_bytes": alg_step,
        "wall_s_timed": t1 - t0,
        "phase_ms_per_step": {k: v["ms_total"] / nprof for k, v in phase.items()},
        "phase_note": "untimed pass of %d steps with events around every launch" % nprof,
        "fp16_rejected_in_fp32": info.stat_fp32_pairs, "fp64_tier_pairs": info.stat_fp64_pairs,
    }
    if not args.no_extras:
        line["fp64_cll"] = bench_fp64(sph, ps, xyz, dev, stream, max(3, args.steps // 4), value)
        line["fp64_cll"]["device_fp64_fma_tflops"] = sph.sph_device_fp64_rate() / 1e12
        line["e2e"] = bench_e2e(sph, ps, dev, stream, args)
        if world > 1:
            e = torch.tensor([line["e2e"]["seconds"]], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(e, op=torch.distributed.ReduceOp.MAX)
            line["e2e"]["value"] = world * n * args.steps / float(e.item())
        line["e2e"].pop("seconds", None)
        if world == 1 and rank == 0:
            line["cpu_baseline"] = cpu_baseline(ps)
    sph.sph_grid_free(grid)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_fp64(sph, ps, xyz, dev, stream, steps, fp16_value):
    """The FP64 cell link-list on the same GPU, same binning and CSR."""
    import torch
    n = ps.n
    sptr = stream.cuda_stream
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL, precision=sph.SPH_PREC_FP64_CLL)
    g = sph.sph_bin_cells(params, xyz, n, sptr, None)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = sph.sph_nnps_query(g, rp, None, 0, True, None, sptr)
    col = torch.empty(nnz + 1024, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        sph.sph_bin_cells(params, xyz, n, sptr, g)
        sph.sph_nnps_query(g, rp, col, col.numel(), False, rho, sptr)

    step()
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    sph.sph_grid_check(g, sptr)
    sph.sph_grid_free(g)
    v = n * steps / (sum(ms) / 1e3)
    return {"value": v, "unit": "particles/s", "ms_per_step": sum(ms) / steps, "steps": steps,
            "fp16_rcll_speedup": fp16_value / v}


def bench_e2e(sph, ps, dev, stream, args):
    """Through the host-buffer C-ABI call: pinned host coordinates in, density
    and nnz out, every step (H2D and D2H inside the timed region)."""
    import torch
    n = ps.n
    sptr = stream.cuda_stream
    xyz_h = torch.from_numpy(ps.xyz).pin_memory()
    rho_h = torch.empty(n, dtype=torch.float32).pin_memory()
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    g, nnz = sph.sph_search_host(params, xyz_h, n, rho_h, sptr, None)
    for _ in range(2):
        sph.sph_search_host(params, xyz_h, n, rho_h, sptr, g)
    torch.cuda.synchronize()
    t = 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        sph.sph_search_host(params, xyz_h, n, rho_h, sptr, g)
        t += time.perf_counter() - t0
    sph.sph_grid_free(g)
    return {"value": n * args.steps / t, "unit": "particles/s", "h2d_bytes_per_step": n * ps.dim * 8,
            "d2h_bytes_per_step": n * 4 + 8, "seconds": t}


if __name__ == "__main__":
    sys.exit(main())
