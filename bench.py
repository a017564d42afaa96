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
    ap.add_argument("--workload", choices=["3d_1m", "2d_10k", "3d_8m", "batch_256", "serve"], default="3d_1m")
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
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2401_08586_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name, kernel_tag, key="bytes_per_launch"):
    """DRAM bytes (or, key="inst_per_launch", warp instructions) per launch of
    the dominant kernel from the committed ncu summary, only if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload_name][kernel_tag]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e[key])
    except Exception:
        return None


KERNEL_SOURCES = ("nnps_tile.cu", "nnps_common.cuh", "sph_internal.cuh", "lookback.cuh", "fastdiv.h", "tile_rows.cuh")


def issue_per_clock(sm_count):
    """Warp instructions a device can issue per clock: 4 schedulers per SM,
    one warp instruction each (Blackwell SM)."""
    return 4 * sm_count


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every SAMPLE_MS ms
    from just before the timed region to just after it."""

    SAMPLE_MS = 10

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
                 "-lms", str(self.SAMPLE_MS)], stdout=self.tmp, stderr=subprocess.DEVNULL)
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
    from paper_2401_08586_gb300 import replicas
    return replicas.rank_env()


# ----------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """FP64 CPU oracle (cell link-list + density) on the host cores."""
    if rank != 0:
        return 0
    import oracle
    threads = os.cpu_count() or 1
    oracle.build.build()
    if args.workload in ("batch_256", "serve"):
        return run_reference_systems(args, threads)
    ps, desc = workload(args.workload)

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
        "config": workload_config(desc, ps, world),
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": threads, "kind": "oracle",
                         "sample": "full workload per step (FP64 cell link-list + density, OpenMP rows)"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(desc, ps, world):
    """The bench line's `config`, the same for both arms (the workload, its
    size and the output form; L2 handling of the GPU arm's timing)."""
    return {"workload": desc, "n_particles": ps.n, "dim": ps.dim, "order": "cell",
            "density": "fused, fp32 accumulation", "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference_systems(args, threads):
    """Reference arm of the batched and served workloads: the oracle over a
    bounded sample of their systems (batched: the first systems in order;
    served: the first requests, one after another, no queueing)."""
    import numpy as np
    import oracle
    from paper_2401_08586_gb300 import workloads as W
    if args.workload == "batch_256":
        systems = W.c4_batched()
        desc = BATCH_DESC
    else:
        systems = [W.materialise_request(sp) for _, sp, _ in W.c5_request_stream(count=40, materialise=False)]
        desc = SERVE_DESC % (len(systems), 0)
    per = []
    for ps in systems:
        t0 = time.perf_counter()
        rp, col = oracle.cll(ps.xyz, ps.kh, threads=threads)
        oracle.density(ps.xyz, ps.h, rp, col, threads=threads)
        per.append((ps.n, time.perf_counter() - t0))
        if sum(t for _, t in per) > 20.0:
            break
    parts = sum(n for n, _ in per)
    tot = sum(t for _, t in per)
    sample = "first %d of %d systems (%d particles), FP64 cell link-list + density" % (len(per), len(systems), parts)
    if args.workload == "serve":
        lat = np.array([1e3 * t for _, t in per])
        value, unit, hib = float(np.percentile(lat, 99)), "ms", False
    else:
        value, unit, hib = parts / tot, "particles/s", True
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": len(per),
            "warmup": 0, "ms_per_step": 1e3 * tot / len(per), "higher_is_better": hib, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    from paper_2401_08586_gb300 import replicas
    if world > 1:
        torch.cuda.set_device(local)
        replicas.init("nccl", world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2401_08586_gb300 import sph

    sph.load(build_if_missing=True)
    if args.workload == "batch_256":
        return bench_batch(args, sph, dev, world, rank, local)
    if args.workload == "serve":
        return bench_serve_line(args, sph, dev, world, rank, local)
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
        replicas.barrier(world)
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
    dev_total_s = replicas.max_over_ranks(sum(step_ms) / 1e3, world, dev)
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
                "traffic": None}
    # the committed figures are per launch over 1,000,000 particles (the
    # recipe at side 100); other sides scale with the particle count
    per_m = n / 1.0e6
    traffic = ncu_traffic(args.workload, dom)
    if traffic is not None:
        roofline["traffic"] = traffic * per_m
    # the bound that applies to the search: instruction issue (measured warp
    # instructions per launch from the committed capture, scaled to this
    # workload, over the event-timed launch, against the issue rate at the SM
    # clock sampled during the timed region)
    clocks = clk.summary()
    inst = ncu_traffic(args.workload, dom, "inst_per_launch")
    inst = None if inst is None else inst * per_m
    issue = None
    if inst is not None and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ipeak = issue_per_clock(sms) * clocks["sm_mhz"] * 1e6
        ia = inst / (dom_ms * 1e-3)
        issue = {"bound": "issue", "kernel": roofline["kernel"], "achieved": ia, "peak": ipeak,
                 "unit": "warp-instructions/s", "frac": ia / ipeak, "inst_per_launch": inst,
                 "peak_source": "%d SMs (device properties) x 4 schedulers x 1 warp-instruction/clock x "
                                "sampled SM clock" % sms}
    # whole path: binning 56 B/particle, search + fused density 36 B/particle + 4 B/neighbour
    alg_step = n * (56 + 36) + 4 * nnz
    step_ms_mean = 1e3 * dev_total_s / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms_mean, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": workload_config(desc, ps, world),
        "clocks": clocks,
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_issue": issue,
        "nnz": nnz, "neighbours_per_particle": nnz / n,
        "step_hbm_frac": alg_step / (step_ms_mean * 1e-3) / 1e9 / peak,
        "step_algorithmic_bytes": alg_step,
        "wall_s_timed": t1 - t0,
        "phase_ms_per_step": {k: v["ms_total"] / nprof for k, v in phase.items()},
        "phase_note": "untimed pass of %d steps with events around every launch" % nprof,
        "fp16_rejected_in_fp32": info.stat_fp32_pairs, "fp64_tier_pairs": info.stat_fp64_pairs,
    }
    if not args.no_extras:
        line["fp64_cll"] = bench_fp64(sph, ps, xyz, dev, stream, max(3, args.steps // 4), value,
                                      line.get("roofline", {}).get("launch_ms"))
        line["fp64_cll"]["device_fp64_fma_tflops"] = sph.sph_device_fp64_rate() / 1e12
        line["query_variants"] = bench_query_variants(sph, ps, xyz, dev, stream, max(3, min(args.steps, 20)))
        if args.workload == "3d_1m" and SIDE == 100:
            line["c3_8m"] = bench_c3(sph, dev, stream, max(3, min(args.steps, 10)), peak, peak_src)
            line["c4_batch"] = bench_c4(sph, dev, stream, max(3, min(args.steps, 10)), peak, peak_src)
        line["e2e"] = bench_e2e(sph, ps, dev, stream, args)
        if world > 1:
            line["e2e"]["value"] = world * n * args.steps / replicas.max_over_ranks(line["e2e"]["seconds"], world,
                                                                                    dev)
        line["e2e"].pop("seconds", None)
        line["gradient_a5"] = bench_gradient(sph, ps, xyz, grid, row_ptr, col, dev, stream, args.steps)
        line["density_half"] = bench_density_half(sph, ps, grid, dev, stream, args.steps)
        line["half_stencil_csr"] = bench_half_csr(sph, ps, xyz, dev, stream, max(3, min(args.steps, 10)),
                                                  line["roofline"]["launch_ms"])
        line["timestep"] = bench_timestep(sph, ps, xyz, dev, stream, row_ptr, col, cap, rho, args.steps)
        line["serving"] = bench_serve(sph, dev, count=2000, warm=200)
        if world == 1 and rank == 0:
            line["cpu_baseline"] = cpu_baseline(ps)
    sph.sph_grid_free(grid)
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish(world)
    return 0


def bench_fp64(sph, ps, xyz, dev, stream, steps, fp16_value, fp16_search_ms=None):
    """The FP64 cell link-list on the same GPU, same binning and CSR: the tile
    search with the FP64 test and FP64 density (the same kernel structure as
    the FP16-RCLL search, so the ratio is one of precision), and, as a second
    figure, the two-pass CTA-per-cell FP64 search."""
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

    def timed(k_steps):
        step()
        torch.cuda.synchronize()
        ms = []
        for k in range(k_steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / k_steps

    sph.sph_profile_reset()
    sph.sph_profile_select("fused")
    sph.sph_profile_enable(True)
    t_tile = timed(steps)
    sph.sph_profile_enable(False)
    fms, fc = sph.sph_profile_read("fused")
    search_ms = fms / fc if fc else None
    sph.sph_grid_set_option(g, sph.SPH_OPT_FUSED, 0)
    t_two = timed(max(2, steps // 3))
    sph.sph_grid_check(g, sptr)
    sph.sph_grid_free(g)
    v = n / (t_tile / 1e3)
    out = {"value": v, "unit": "particles/s", "ms_per_step": t_tile, "steps": steps,
           "search": "single-pass tile search, FP64 test and FP64 density (same tiles, cull, look-back, CSR)",
           "search_ms": search_ms, "fp16_rcll_speedup": fp16_value / v,
           "two_pass_ms_per_step": t_two,
           "two_pass_note": "FP64 two-pass search, one thread block per cell (the earlier baseline)"}
    if fp16_search_ms and search_ms:
        out["search_speedup"] = search_ms / fp16_search_ms
    return out


def bench_c4(sph, dev, stream, steps, peak, peak_src):
    """The batched workload (C4: 256 independent 3D systems of 2e3..2e5
    particles) through sph_batch_run: per run the bounds, then one replayed
    CUDA graph (binning, tile list, persistent search); CUDA events per run,
    the search launch timed in an untimed pass of direct launches."""
    import torch
    from paper_2401_08586_gb300 import workloads as W
    systems = W.c4_batched()
    xs = [torch.from_numpy(ps.xyz).to(dev) for ps in systems]
    params = [sph.make_params(3, ps.h, ps.kh, order=sph.SPH_ORDER_CELL) for ps in systems]
    ntot = sum(ps.n for ps in systems)
    pairs = list(zip(xs, params))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    b = sph.Batch()
    for _ in range(3):
        flush.fill_(1.0)
        b.run(pairs, stream=stream)
    torch.cuda.synchronize()
    st0 = b.stats()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rp, col, rho, orig, first = b.run(pairs, stream=stream)
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    st = b.stats()
    nnz = int(rp[-1].item())
    b.set_option(sph.SPH_BATCH_OPT_GRAPH, 0)
    sph.sph_profile_reset()
    sph.sph_profile_select("fused")
    for k in range(3):
        flush.fill_(float(k))
        b.run(pairs, stream=stream)
    torch.cuda.synchronize()
    sph.sph_profile_enable(False)
    fms, fc = sph.sph_profile_read("fused")
    b.close()
    t = sum(ms) / steps
    launch = fms / max(fc, 1)
    alg = ntot * (8 + 16 + 8 + 4) + 4 * nnz
    return {"workload": BATCH_DESC, "n_particles": ntot, "systems": len(systems), "value": ntot / (t * 1e-3),
            "unit": "particles/s", "ms_per_run": t, "steps": steps, "nnz": nnz,
            "graph_replays": st.graph_replays - st0.graph_replays, "direct_launches_per_run": st.direct_launches,
            "roofline": {"bound": "hbm", "kernel": "k_nnps_tile (batch)", "achieved": alg / (launch * 1e-3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": alg / (launch * 1e-3) / 1e9 / peak,
                         "peak_source": peak_src, "launch_ms": launch, "algorithmic_bytes_per_launch": alg}}


def bench_half_csr(sph, ps, xyz, dev, stream, steps, full_search_ms):
    """The neighbour list over a half stencil (sph_nnps_query_half: each pair
    decided once and written into both rows, then a per-row sort) on the
    step's workload, with the fused density: CUDA events around the call (it
    reads nnz back to size the fill, so the figure includes that round trip)
    and the library's kernel times; beside it the tile search's launch."""
    import torch
    n = ps.n
    sptr = stream.cuda_stream
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    g = sph.sph_bin_cells(params, xyz, n, sptr, None)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = sph.sph_nnps_query_half(g, rp, None, 0, None, sptr)
    col = torch.empty(nnz + 1024, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sph.sph_nnps_query_half(g, rp, col, col.numel(), rho, sptr)
    torch.cuda.synchronize()
    sph.sph_profile_reset()
    sph.sph_profile_select(None)
    sph.sph_profile_enable(True)
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sph.sph_nnps_query_half(g, rp, col, col.numel(), rho, sptr)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    sph.sph_profile_enable(False)
    kern = {}
    for tag in ("count", "scan", "fill", "sort"):
        kms, c = sph.sph_profile_read(tag)
        if c:
            kern[tag] = kms / steps
    sph.sph_grid_free(g)
    t = sum(ms) / steps
    return {"ms": t, "kernel_ms": kern, "tile_search_ms": full_search_ms,
            "slower_than_tile_search": t / full_search_ms if full_search_ms else None,
            "note": "each pair decided once (13 of 26 neighbour cells), written into both rows, rows sorted; "
                    "fused density with atomic partner shares"}


def bench_c3(sph, dev, stream, steps, peak, peak_src):
    """The 8M non-uniform dam-break set (C3): the same step (binning + tile
    search with fused density, cell order), CUDA events per step, the search
    launch timed by the library's events and its HBM roofline (36 B per
    particle + 4 B per neighbour)."""
    import torch
    from paper_2401_08586_gb300 import workloads as W
    ps = W.c3_3d_dambreak()
    n = ps.n
    sptr = stream.cuda_stream
    xyz = torch.from_numpy(ps.xyz).to(dev)
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    g = sph.sph_bin_cells(params, xyz, n, sptr, None)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = sph.sph_nnps_query(g, rp, None, 0, True, None, sptr)
    col = torch.empty(nnz + 1024, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        sph.sph_bin_cells(params, xyz, n, sptr, g)
        sph.sph_nnps_query(g, rp, col, col.numel(), False, rho, sptr)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    sph.sph_profile_reset()
    sph.sph_profile_select("fused")
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    sph.sph_profile_enable(False)
    fms, fc = sph.sph_profile_read("fused")
    sph.sph_grid_check(g, sptr)
    sph.sph_grid_free(g)
    t = sum(ms) / steps
    launch = fms / fc
    alg = n * (8 + 16 + 8 + 4) + 4 * nnz
    achieved = alg / (launch * 1e-3) / 1e9
    return {"workload": "3d_8m_dambreak: 200^3 lattice dx=1/200 in z<1 of a 1x1x2 box, 5% spray in z in (1,2], "
                        "jitter U(+-0.2dx), h=1.5dx, kh=3dx, seed 3",
            "n_particles": n, "value": n / (t * 1e-3), "unit": "particles/s", "ms_per_step": t, "steps": steps,
            "nnz": nnz, "neighbours_per_particle": nnz / n,
            "roofline": {"bound": "hbm", "kernel": "k_nnps_tile", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "launch_ms": launch,
                         "algorithmic_bytes_per_launch": alg}}


def bench_query_variants(sph, ps, xyz, dev, stream, steps):
    """The search's other query forms on the same workload, each through the
    tile search: count only (col == NULL: row pointers and nnz, the capacity
    discovery) and canonical order (input-order rows, input-index columns
    ascending: cell-order search, then row permutation and per-row sort).
    CUDA events around each call; the canonical query reads nnz back to the
    host inside the call, so its figure includes that round trip, and the
    library's kernel times are given beside it."""
    import torch
    n = ps.n
    sptr = stream.cuda_stream
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}

    def events(fn, k_steps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(k_steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / k_steps

    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    g = sph.sph_bin_cells(params, xyz, n, sptr, None)
    out["count_only_ms"] = events(lambda: sph.sph_nnps_query(g, rp, None, 0, False, None, sptr), steps)
    sph.sph_grid_free(g)

    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CANONICAL)
    g = sph.sph_bin_cells(params, xyz, n, sptr, None)
    nnz = sph.sph_nnps_query(g, rp, None, 0, True, None, sptr)
    col = torch.empty(nnz + 1024, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    sph.sph_profile_reset()
    sph.sph_profile_select(None)
    sph.sph_profile_enable(True)
    out["canonical_ms"] = events(lambda: sph.sph_nnps_query(g, rp, col, col.numel(), False, rho, sptr), steps)
    sph.sph_profile_enable(False)
    kern = {}
    for tag in ("scan", "fused", "canon", "sort"):
        ms, c = sph.sph_profile_read(tag)
        if c:
            kern[tag] = ms / (steps + 1)
    out["canonical_kernel_ms"] = kern
    sph.sph_grid_check(g, sptr)
    sph.sph_grid_free(g)
    return out


def bench_gradient(sph, ps, xyz, grid, row_ptr, col, dev, stream, steps):
    """The Appendix Eq. A5 gradient of f = x^3 over the step's CSR (the
    paper's second timed kernel), CUDA events on the stream."""
    import torch
    f = (xyz[:, 0] ** 3).contiguous()
    # the grid's last query wrote row_ptr / col in cell order
    out = torch.empty((ps.n, ps.dim), dtype=torch.float64, device=dev)
    sptr = stream.cuda_stream
    ms = []
    for k in range(steps + 3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sph.sph_gradient_a5(grid, row_ptr, col, f, out, sptr)
        b.record(stream)
        b.synchronize()
        if k >= 3:
            ms.append(a.elapsed_time(b))
    t = sum(ms) / len(ms)
    return {"ms": t, "particles_per_s": ps.n / (t * 1e-3), "field": "x^3"}


def bench_density_half(sph, ps, grid, dev, stream, steps):
    """The summation density over the half stencil (no neighbour list) on
    the step's grid, CUDA events on the stream, L2 flushed between calls."""
    import torch
    rho = torch.empty(ps.n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sptr = stream.cuda_stream
    ms = []
    for k in range(steps + 3):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sph.sph_density_half(grid, rho, sptr)
        b.record(stream)
        b.synchronize()
        if k >= 3:
            ms.append(a.elapsed_time(b))
    t = sum(ms) / len(ms)
    return {"ms": t, "particles_per_s": ps.n / (t * 1e-3),
            "note": "density only (no CSR); the search with CSR and fused density is roofline.launch_ms"}


def bench_timestep(sph, ps, xyz, dev, stream, row_ptr, col, cap, rho, steps):
    """One SPH time step's search through the Eq. 8-9 update (sph_advance +
    query) against re-binning the moved positions (sph_bin_cells + query).
    The particles move back and forth by a random displacement of up to
    0.15 dx per axis, so about a fifth of them change cell every step."""
    import torch
    sptr = stream.cuda_stream
    n = ps.n
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    v = (torch.rand(xyz.shape, generator=g, device=dev, dtype=torch.float64) * 2 - 1) * (0.15 * ps.dx)
    xs = [xyz, xyz + v]
    vs = [-v, v]
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        ms = []
        for k in range(steps + 3):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(k)
            b.record(stream)
            b.synchronize()
            if k >= 3:
                ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms)

    grid = sph.sph_bin_cells(params, xs[0], n, sptr, None)

    def adv(k):
        sph.sph_advance(grid, xs[(k + 1) % 2], vs[(k + 1) % 2], 1.0, sptr)
        sph.sph_nnps_query(grid, row_ptr, col, cap, False, rho, sptr)

    def rebin(k):
        sph.sph_bin_cells(params, xs[(k + 1) % 2], n, sptr, grid)
        sph.sph_nnps_query(grid, row_ptr, col, cap, False, rho, sptr)

    ms_adv = timed(adv)
    sph.sph_bin_cells(params, xs[0], n, sptr, grid)
    ms_bin = timed(rebin)
    sph.sph_grid_check(grid, sptr)
    sph.sph_grid_free(grid)
    return {"advance_plus_query_ms": ms_adv, "rebin_plus_query_ms": ms_bin,
            "advance_particles_per_s": n / (ms_adv * 1e-3), "displacement": "U(+-0.15 dx) per axis, back and forth"}


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
    # pipelined: two grids on two streams, each step still copies its inputs
    # in and its density and nnz out, but one step's copies and host work run
    # while the other step's kernels do (sph_search_host_async / _finish)
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    xs_h = [xyz_h, torch.from_numpy(ps.xyz).pin_memory()]
    rhos_h = [rho_h, torch.empty(n, dtype=torch.float32).pin_memory()]
    gp = [None, None]
    for b in range(2):  # first calls size the grid-owned CSR (synchronous)
        gp[b] = sph.sph_search_host_async(params, xs_h[b], n, rhos_h[b], streams[b].cuda_stream, None)
        sph.sph_search_host_finish(gp[b])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        b = k & 1
        if k >= 2:
            sph.sph_search_host_finish(gp[b])
        sph.sph_search_host_async(params, xs_h[b], n, rhos_h[b], streams[b].cuda_stream, gp[b])
    nnz_p = [sph.sph_search_host_finish(gp[b]) for b in range(2)]
    t_pipe = time.perf_counter() - t0
    for b in range(2):
        sph.sph_grid_free(gp[b])
    assert nnz_p[0] == nnz_p[1] == nnz
    # the same with the whole CSR copied back to pinned host memory as well
    rp_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    col_h = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
    steps_csr = max(3, args.steps // 4)
    t_csr = 0.0
    for k in range(steps_csr):
        t0 = time.perf_counter()
        _, nnz_k = sph.sph_search_host(params, xyz_h, n, rho_h, sptr, g)
        sph.sph_grid_csr_copy(g, rp_h, col_h, sptr)
        t_csr += time.perf_counter() - t0
    sph.sph_grid_free(g)
    return {"value": n * args.steps / t_pipe, "unit": "particles/s", "h2d_bytes_per_step": n * ps.dim * 8,
            "d2h_bytes_per_step": n * 4 + 8, "seconds": t_pipe,
            "how": "sph_search_host_async / sph_search_host_finish on two grids and streams: every step copies its "
                   "coordinates in from pinned host memory and its density and nnz out; one step's copies overlap "
                   "the other's kernels",
            "serial": {"value": n * args.steps / t, "unit": "particles/s",
                       "note": "sph_search_host, one call per step, synchronised"},
            "with_csr": {"value": n * steps_csr / t_csr, "unit": "particles/s", "steps": steps_csr,
                         "h2d_bytes_per_step": n * ps.dim * 8,
                         "d2h_bytes_per_step": n * 4 + 8 + (n + 1) * 8 + nnz * 4,
                         "note": "sph_search_host, then sph_grid_csr_copy of row_ptr and col to pinned host memory"}}


SERVE_DESC = ("serve: Poisson arrivals at 200 req/s, 70%% 3D / 30%% 2D, N log-uniform in [1e3, 2e6], jittered "
              "lattices dx = 1/ceil(N^(1/d)), h/dx U[1.2, 1.5], kh = 2h, 64 GB budget, 4 worker streams, seed 5; "
              "%d timed requests after %d warm-up")


def device_request(spec, dev):
    """One request's coordinates drawn on the device (the lattice recipe of
    the request stream, jitter from torch's generator seeded by the request)."""
    import torch
    dim, n = spec["dim"], spec["n"]
    side = int(math.ceil(n ** (1.0 / dim)))
    dx = 1.0 / side
    idx = torch.arange(n, device=dev, dtype=torch.int64)
    cols = []
    for k in range(dim):
        cols.append(((idx // side ** k) % side).to(torch.float64).add_(0.5).mul_(dx))
    xyz = torch.stack(cols, 1)
    g = torch.Generator(device=dev)
    g.manual_seed(spec["seed"] % (1 << 62))
    xyz += (torch.rand(xyz.shape, generator=g, device=dev, dtype=torch.float64) * 2 - 1) * (0.1 * dx)
    return xyz.contiguous(), spec["hr"] * dx


def bench_serve(sph, dev, count=2000, warm=200, rate=200.0):
    """Replay the request stream against a server; latencies of the requests
    after the warm-up.  Results stay on the device until each is released;
    the D2H figure adds each result's copy to pinned host memory."""
    import threading
    import numpy as np
    import torch
    from paper_2401_08586_gb300 import workloads as W
    specs = W.c5_request_stream(count=count + warm, rate=rate, materialise=False)
    reqs = [device_request(sp, dev) for _, sp, _ in specs]
    torch.cuda.synchronize()
    srv = sph.Server(64 << 30, streams=4)
    tickets = [None] * len(specs)
    done = {}
    d2h_s = {}
    pin_col = torch.empty(2_000_000 * 130, dtype=torch.int32).pin_memory()
    pin_rp = torch.empty(2_000_001, dtype=torch.int64).pin_memory()
    pin_rho = torch.empty(2_000_000, dtype=torch.float32).pin_memory()
    copy_stream = torch.cuda.Stream(dev)
    ready = threading.Event()
    failed = {}

    def completer():
        for k in range(len(specs)):
            while tickets[k] is None:
                ready.wait(0.001)
            res = srv.wait(tickets[k])
            if res.status != sph.SPH_OK:
                failed[k] = "%d: %s" % (res.status, sph.sph_last_error())
                srv.release(tickets[k])
                continue
            t0 = time.perf_counter()
            sph.sph_result_copy(srv.handle, tickets[k], pin_rp, pin_col, pin_rho, None, copy_stream)
            copy_stream.synchronize()
            d2h_s[k] = time.perf_counter() - t0
            done[k] = (res.t_submit_ns, res.t_admit_ns, res.t_done_ns, res.n)
            srv.release(tickets[k])

    th = threading.Thread(target=completer)
    th.start()
    t_start = time.perf_counter()
    for k, (t_arr, sp, _) in enumerate(specs):
        now = time.perf_counter() - t_start
        if t_arr > now:
            time.sleep(t_arr - now)
        xyz, h = reqs[k]
        tickets[k] = srv.submit(xyz, sph.make_params(sp["dim"], h, 2 * h, order=sph.SPH_ORDER_CELL))
        ready.set()
    th.join()
    st = srv.stats()
    srv.close()
    if failed:
        raise RuntimeError("%d requests failed, first: %s" % (len(failed), next(iter(failed.items()))))
    ks = range(warm, len(specs))
    lat = np.array([(done[k][2] - done[k][0]) / 1e6 for k in ks])
    lat_d2h = np.array([(done[k][2] - done[k][0]) / 1e6 + 1e3 * d2h_s[k] for k in ks])
    queue = np.array([(done[k][1] - done[k][0]) / 1e6 for k in ks])
    parts = sum(done[k][3] for k in ks)
    span_s = (max(done[k][2] for k in ks) - min(done[k][0] for k in ks)) / 1e9
    return {"requests": count, "warmup": warm, "rate_per_s": rate,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p99_with_d2h_ms": float(np.percentile(lat_d2h, 99)), "mean_ms": float(lat.mean()),
            "p99_queue_ms": float(np.percentile(queue, 99)), "particles_per_s": parts / span_s,
            "batches": int(st.batches), "batched_requests": int(st.batched_requests),
            "peak_held_gb": st.peak_held_bytes / 2 ** 30}


def bench_serve_line(args, sph, dev, world, rank, local):
    count = args.steps if args.steps != 100 else 2000
    with ClockSampler(local) as clk:
        r = bench_serve(sph, dev, count=count, warm=200)
    line = {"metric": METRIC, "value": r["p99_ms"], "unit": "ms", "n_gpus": world, "steps": count,
            "warmup": 200, "ms_per_step": r["mean_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": SERVE_DESC % (count, 200), "parallelism": "replicas" if world > 1 else "single"},
            "clocks": clk.summary(), "serving": r}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


BATCH_DESC = ("batch_256: 256 independent 3D jittered lattices, N log-uniform in [2e3, 2e5], dx U[0.005, 0.02], "
              "h/dx U[1.2, 1.5], kh = 2h, jitter U(+-0.1dx), seed 4")


def bench_batch(args, sph, dev, world, rank, local):
    """The batched workload through sph_batch_run: one step = one run over all
    256 systems (bounds, binning, tile search with fused density, nnz read)."""
    import torch
    from paper_2401_08586_gb300 import replicas
    from paper_2401_08586_gb300 import workloads as W
    all_systems = W.c4_batched()
    systems = replicas.shard(all_systems, world, rank)  # independent systems: round-robin over the ranks
    xs = [torch.from_numpy(ps.xyz).to(dev) for ps in systems]
    params = [sph.make_params(3, ps.h, ps.kh, order=sph.SPH_ORDER_CELL) for ps in systems]
    ntot = sum(ps.n for ps in systems)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    b = sph.Batch()
    pairs = list(zip(xs, params))
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        b.run(pairs, stream=stream)
    torch.cuda.synchronize()
    st0 = b.stats()
    sph.sph_profile_reset()
    sph.sph_profile_select("fused")
    launches0 = sph.sph_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        replicas.barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            rp, col, rho, orig, first = b.run(pairs, stream=stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        replicas.barrier(world)
        t1 = time.perf_counter()
    launches = sph.sph_launch_count() - launches0
    sph.sph_profile_enable(False)
    st = b.stats()
    # the search runs inside the replayed graph, where no per-launch events are
    # recorded: its launch time comes from an untimed pass of direct launches
    b.set_option(sph.SPH_BATCH_OPT_GRAPH, 0)
    sph.sph_profile_reset()
    sph.sph_profile_select("fused")
    for k in range(3):
        flush.fill_(float(k))
        b.run(pairs, stream=stream)
    torch.cuda.synchronize()
    sph.sph_profile_enable(False)
    ms, c = sph.sph_profile_read("fused")
    b.set_option(sph.SPH_BATCH_OPT_GRAPH, 1)
    total_s = sum(a.elapsed_time(e) for a, e in evs) / 1e3
    nnz = int(rp[-1].item())
    value = replicas.whole_job_rate(ntot * args.steps, total_s, world, dev)
    dom_ms = ms / max(c, 1)
    alg = ntot * (8 + 16 + 8 + 4) + 4 * nnz
    peak, peak_src = measured_peaks()
    achieved = alg / (dom_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "n_particles": int(replicas.sum_over_ranks(ntot, world, dev)),
                   "systems": len(all_systems), "dim": 3, "order": "cell",
                   "density": "fused, fp32 accumulation", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clk.summary(), "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "k_nnps_tile (batch)", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "launch_ms": dom_ms,
                     "algorithmic_bytes_per_launch": alg, "traffic": None},
        "nnz": nnz, "neighbours_per_particle": nnz / ntot, "wall_s_timed": t1 - t0,
        "batch": {"graph_replays_timed": st.graph_replays - st0.graph_replays, "graph_captures": st.graph_captures,
                  "graph_holds": "binning, tile list, counter reset and the persistent tile search",
                  "direct_launches_last_run": st.direct_launches,
                  "tuned_staging_bytes": st.tuned_staging, "fp32_pairs": st.fp32_pairs, "fp64_pairs": st.fp64_pairs},
    }
    if not args.no_extras:
        # end to end: pinned host coordinates in, densities and nnz out, every step
        xh = [torch.from_numpy(ps.xyz).pin_memory() for ps in systems]
        rho_h = torch.empty(ntot, dtype=torch.float32).pin_memory()
        xd = [torch.empty_like(x) for x in xs]
        pd = list(zip(xd, params))
        for x, h in zip(xd, xh):
            x.copy_(h, non_blocking=True)
        b.run(pd, stream=stream)
        torch.cuda.synchronize()
        t = 0.0
        for k in range(args.steps):
            ta = time.perf_counter()
            for x, h in zip(xd, xh):
                x.copy_(h, non_blocking=True)
            rp, col, rho, orig, first = b.run(pd, stream=stream)
            rho_h.copy_(rho, non_blocking=True)
            torch.cuda.synchronize()
            t += time.perf_counter() - ta
        line["e2e"] = {"value": ntot * args.steps / t, "unit": "particles/s", "h2d_bytes_per_step": ntot * 3 * 8,
                       "d2h_bytes_per_step": ntot * 4 + 8}
        if world == 1 and rank == 0:
            line["cpu_baseline"] = cpu_baseline_systems(systems)
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish(world)
    return 0


def cpu_baseline_systems(systems, budget_s=12.0):
    """The oracle on all host cores over the batch's systems in order, until
    about budget_s has passed (a bounded sample of the workload)."""
    import oracle
    oracle.build.build()
    threads = os.cpu_count() or 1
    done, t = 0, 0.0
    k = 0
    while t < budget_s and k < len(systems):
        ps = systems[k]
        t0 = time.perf_counter()
        rp, col = oracle.cll(ps.xyz, ps.kh, threads=threads)
        oracle.density(ps.xyz, ps.h, rp, col, threads=threads)
        t += time.perf_counter() - t0
        done += ps.n
        k += 1
    return {"value": done / t, "unit": "particles/s", "cores": threads, "kind": "oracle",
            "sample": "first %d of %d systems (%d particles), FP64 cell link-list + density" % (k, len(systems), done)}


if __name__ == "__main__":
    sys.exit(main())
