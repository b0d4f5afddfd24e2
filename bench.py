"""Benchmark of the particle-side hot path on GB300.

One step = one fluid step of the coupled loop: 20 DEM substeps (binning and
lists when due, Hertz-Mindlin contact with springs, lubrication, drag /
pressure-gradient / added-mass forces, leapfrog update) followed by one
diffusion-based averaging (fixed-point PCM deposition + implicit smoothing by
Chebyshev iterative refinement), on the large settled bed: 10,000,000 spheres in
a periodic 400 x 200 x 100 mm box on a 256 x 128 x 64 mesh.  Metric:
particle-steps/s = N x substeps / device seconds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun, one rank per GPU) runs one independent bed per rank (weak
scaling, no collective on the data path).  --impl reference times the FP64 CPU
oracle on this host's cores on a bounded sample of the same workload (no GPU).
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (contact+coupling+averaging), % HBM roofline, vs plain form"
UNIT = "particle-steps/s"
SUBSTEPS = 20
WORKLOAD = ("large settled bed: 10,000,000 spheres, d ~ U[0.4, 0.6] mm, rho 2500, settled into a "
            "~14 mm deep bed (FIRE energy-minimised 4 x 4 mm periodic block of 2,000 spheres tiled "
            "100 x 50: ~5 contacts per sphere, packing fraction ~0.6) in a periodic 400x200x100 mm "
            "box, wall z=0, water, 256x128x64 mesh, mean flow 0.3 m/s + Gaussian-filtered noise "
            "(rms 0.03 m/s), DU/Dt = U.grad U; Hertz-Mindlin + lubrication + drag + pressure "
            "gradient + added mass, diffusion averaging b=1.5 mm; step = 20 substeps "
            "(dt=1e-6 s) + 1 averaging")
WORKLOAD_200K = ("sheared sediment bed: 200,000 lognormal spheres (median 0.5 mm, sigma_ln 0.1) "
                 "settled (FIRE energy-minimised 8 x 4 mm block tiled 8 x 8) in a periodic "
                 "64x32x64 mm channel, wall z=0, log-law flow u*=0.02 m/s, 64x32x64 mesh; "
                 "step = 20 substeps + 1 averaging")
# committed ncu summaries holding the DRAM bytes per particle-substep of the pair
# list's substep launch (k_pair_forces + k_substep<gather>) with the kernel source hash
TRAFFIC_LARGE = os.path.join(ROOT, "profiles", "traffic_large10M.md")
TRAFFIC_200K = os.path.join(ROOT, "profiles", "traffic_bed200k.md")
KERNEL_SOURCES = ["paper_1601_03801_gb300/csrc/k_force.cu", "paper_1601_03801_gb300/csrc/fluid.cuh",
                  "paper_1601_03801_gb300/csrc/common.cuh", "paper_1601_03801_gb300/csrc/dd.cuh"]


PAIR_VARIANTS = (8, 9)  # substep variants of the pair list (two kernels per substep)


def substep_kernel_name(variant, form="split"):
    """The kernel(s) the roofline line measures for a substep launch variant."""
    if variant in PAIR_VARIANTS and form != "fp64":
        sched = ", ordered" if variant == 9 else ""
        return f"k_pair_forces<{form}{sched}> + k_substep<{form}, gather>"
    return f"k_substep<{form}>"


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(variant, path, bins=None):
    """DRAM bytes per particle-substep of the pair list's substep launch (pair-force and
    gather kernels) from a committed ncu summary, if it was taken on the current kernel
    source, for this launch variant and these bins (bins per cutoff, storage order);
    None for other launch variants (no summary committed)."""
    if variant not in PAIR_VARIANTS or not os.path.exists(path):
        return None, None
    txt = open(path).read()
    k = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    if not k or k.group(1) != kernel_hash():
        return None, None
    for m in re.finditer(r"traffic: variant=(\d+) bins_per_cutoff=(\d+) bin_order=(\d+) "
                         r"bytes_per_particle_substep=([0-9.eE+-]+)", txt):
        if int(m.group(1)) != variant:
            continue
        if bins is not None and (int(m.group(2)), int(m.group(3))) != tuple(bins):
            continue
        return float(m.group(4)), k.group(1)
    return None, None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(total_ms_local, particles_local, steps, world, device="cpu"):
    """Whole-job throughput over ranks: every rank ran its own bed for `steps`
    steps; the job time is the slowest rank's (max over ranks)."""
    total_ms = float(total_ms_local)
    parts = float(particles_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        p = torch.tensor([parts], dtype=torch.float64, device=device)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
        parts = float(p.item())
    value = parts * SUBSTEPS * steps / (total_ms / 1e3)
    return value, total_ms


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def algorithmic_bytes(kbar, cbar, cells, n, form="split"):
    """Algorithmic DRAM bytes of one particle-substep (contact + coupling + update):
    own state x, v, omega read and written (FP64: 3 x 24 x 2 = 144 B), radius and
    lagged acceleration read (16 B), acceleration written (12 B), 4 B per listed
    neighbour index, 24 B per contact spring read plus 12 B owner write, and ~40 B of
    mesh fields per cell shared by C/N spheres.  The plain FP32 form carries FP32
    state and springs: 72 + 16 + 12 + 4 kbar + 18 cbar + 40 C/N."""
    if form == "plain":
        return 72 + 16 + 12 + 4 * kbar + 18 * cbar + 40.0 * cells / n
    if form == "fp64":  # FP64 mesh words too
        return 144 + 16 + 12 + 4 * kbar + 36 * cbar + 80.0 * cells / n
    return 144 + 16 + 12 + 4 * kbar + 36 * cbar + 40.0 * cells / n


def implementation_bytes(kbar, cbar, cells, n):
    """Bytes the split form's layout moves per particle-substep: 32-byte double-float
    records (position + radius, velocity + mass, spin) read and written (96 + 96),
    acceleration and build position (16 + 16), wall mask and list count (8), 4 B per
    listed index, a 32-byte spring record read and written per contact side (64 per
    contact, i.e. 48 per contact and particle with the pair list's single store), and
    two 16-byte mesh words per cell."""
    return 264 + 4 * kbar + 48 * cbar + 32.0 * cells / n


def list_stats(g, n):
    off, _ = g.neighbors()
    ij, _ = g.contacts()
    return float(off[-1]) / n, 2.0 * len(ij) / n


def measure(prm, parts, fl, form, steps, warmup, settle, stream, flush=None, profile=0,
            world=1, local=0, clocks=False):
    """One handle on the workload: untimed settling, W warm-up steps, then K timed
    steps (20 substeps + 1 averaging each) with CUDA events on the launching stream.
    Returns the handle and the measurements."""
    import torch

    from paper_1601_03801_gb300 import sedi

    g = sedi.Sedi(dict(prm, precision_form=form, use_graphs=1, profile=profile), stream=stream)
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.set_fluid(U=fl["U"], DUDt=fl.get("DUDt"))
    g.average_inplace()  # the drag sees a smoothed solid fraction from the start
    for _ in range(settle):
        g.step(SUBSTEPS)
        g.average_inplace()
    for _ in range(warmup):
        g.step(SUBSTEPS)
        g.average_inplace()
    g.sync()
    t0 = g.timings() if profile else None
    st0 = g.stats()
    evs = []
    clk = Clocks(local) if clocks else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clk:
        clk.start()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            if flush is not None:
                flush.zero_()  # L2 flushed between timed steps, outside the events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        g.step(SUBSTEPS)
        g.average_inplace()
        with torch.cuda.stream(stream):
            e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    out = {"clocks": clk.stop() if clk else None,
           "ms": [a.elapsed_time(b) for a, b in evs],
           "stats0": st0, "stats1": g.stats()}
    if profile:
        t1 = g.timings()
        out["phases"] = {k: round((t1[k] - t0[k]) / steps, 4) for k in
                         ("rebuild_ms", "substep_ms", "deposit_ms", "smooth_ms")}
        out["substep_launch_ms"] = ((t1["substep_ms"] - t0["substep_ms"]) /
                                    max(1.0, t1["substep_n"] - t0["substep_n"]))
    return g, out


def roofline(prm, n, g, launch_ms, variant, form="split", traffic=TRAFFIC_LARGE):
    """Roofline of the substep launch: algorithmic bytes (algorithmic_bytes) of every
    particle-substep of one launch / the launch's mean duration (CUDA events inside
    the graph), against the measured HBM copy bandwidth.  `traffic`: the ncu summary
    of this workload's DRAM bytes."""
    kbar, cbar = list_stats(g, n)
    C = int(np.prod(prm["ncell"]))
    alg = algorithmic_bytes(kbar, cbar, C, n, form)
    achieved = alg * n / (launch_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    st = g.stats()
    bins = (st["bins_per_cutoff"], st["bin_order"])
    traffic_pp, _ = measured_traffic(variant, traffic, bins) if form == "split" else (None, None)
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4), "peak_source": peak_kind,
           "traffic": None if traffic_pp is None else round(traffic_pp * n),
           "kernel": substep_kernel_name(variant, form),
           "algorithmic_bytes_per_particle_substep": round(alg, 1),
           "particles_per_launch": n, "launch_ms": round(launch_ms, 5),
           "kbar": round(kbar, 2), "cbar": round(cbar, 2), "cells": C}
    if form == "split":
        out["implementation_bytes_per_particle_substep"] = round(implementation_bytes(kbar, cbar, C, n), 1)
        if traffic_pp is not None:
            out["traffic_bytes_per_particle_substep"] = traffic_pp
            out["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of the launch's two "
                                   "kernels per particle-substep, from the ncu capture of this "
                                   "workload (" + os.path.basename(traffic) + "), times the particles "
                                   "of this launch")
    return out


def tuned_launch(st):
    """The substep launch and bins the autotuner chose (from a handle's stats)."""
    return {"variant": st["substep_variant"], "block": st["substep_block"],
            "bins_per_cutoff": st["bins_per_cutoff"], "bin_order": "xz"[st["bin_order"]] + " fastest",
            "chosen_by": "autotuner"}


def launches_per_step(variant, rebuilds, steps, cells):
    """Kernels of one step: the graph's rebuild check, 20 substeps of one kernel (two
    with the pair list), 16 per list rebuild taken (the split form keeps the pair
    list -- counts, scan, fill -- whatever the variant), then deposition,
    fixed point -> smoothing word, the smoother (the cluster solver: one launch; the
    grid solver: barrier reset + cooperative launch) and the outputs."""
    per_sub = 2 if variant in PAIR_VARIANTS else 1
    per_avg = 4 if cells <= 131072 else 5
    return steps * (1 + per_sub * SUBSTEPS + per_avg) + 16 * rebuilds


def gpu_arm(args):
    import torch

    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import large_case

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prm, parts, fl = large_case()
    n = len(parts["x"])
    C = int(np.prod(prm["ncell"]))
    stream = torch.cuda.Stream()
    # the headline handle runs without per-phase event nodes in its graph; the state
    # (~2 GB) is far larger than L2, so no flush is needed between timed steps
    g, m = measure(prm, parts, fl, "split", args.steps, args.warmup, args.settle, stream,
                   world=world, local=local, clocks=True)
    value, total_ms = aggregate(float(np.sum(m["ms"])), n, args.steps, world, device="cuda")
    st0, st1 = m["stats0"], m["stats1"]
    variant = st1["substep_variant"]
    rebuilds = st1["rebuilds"] - st0["rebuilds"]
    roof = None
    phases = None
    del g
    torch.cuda.empty_cache()
    # phase breakdown and the substep launch time from a second, profiled handle (CUDA
    # events recorded inside the graph around every phase)
    gp, mp = measure(prm, parts, fl, "split", max(3, min(args.steps, 10)), args.warmup, args.settle,
                     stream, profile=1)
    roof = roofline(prm, n, gp, mp["substep_launch_ms"], gp.stats()["substep_variant"])
    phases = mp["phases"]
    gp.close()
    del gp
    torch.cuda.empty_cache()
    e2e = end_to_end(prm, parts, fl, stream, args, world)
    plain = plain_form_leg(prm, parts, fl, stream, args) if rank == 0 and not args.no_plain else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(prm, parts, fl)
    extra = {}
    if rank == 0:
        if not args.no_bed200k:
            extra["bed200k"] = bed200k_leg(args)
        if not args.no_ensemble:
            extra["ensemble"] = ensemble_leg()
        if not args.no_cnn:
            from paper_1601_03801_gb300.workloads import bed_case
            extra["cnn_warm_start"] = cnn_warm_start(*bed_case())
        if not args.no_bounce:
            extra["case1_bounce"] = bounce_leg()

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(total_ms / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 forces; df64 (FP32-pair, 48-bit) state and springs; int64 deposition",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "particles_per_gpu": n, "substeps_per_step": SUBSTEPS,
                           "mesh_cells": C, "form": "split", "graphs": True,
                           "settle_steps_untimed": args.settle,
                           "substep_variant": tuned_launch(st1),
                           "l2": "not flushed: the particle state (~2 GB) is larger than L2",
                           "parallelism": "independent bed per GPU" if world > 1 else "1 GPU"},
                "phases_ms_per_step": phases, "rebuilds_in_timed_region": int(rebuilds),
                "roofline": roof, "e2e": e2e,
                "gpu_launches": int(launches_per_step(variant, rebuilds, args.steps, C)),
                "clocks": m["clocks"], "cpu_baseline": cpu, "other_forms": plain, **extra}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def end_to_end(prm, parts, fl, stream, args, world):
    """The metric through the C ABI with host buffers: every step copies the fluid
    fields (U, grad p, DU/Dt) from pinned host memory to the library, runs 20
    substeps, and averages into pinned host buffers (eps_s, U_s, F_fp), wall clock
    around the steps with the device synchronised on both sides."""
    import torch

    from paper_1601_03801_gb300 import sedi

    n = len(parts["x"])
    C = int(np.prod(prm["ncell"]))
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    Uh = pin(fl["U"])
    gph = pin(np.tile(np.array([0.0, 0.0, -9.81 * 1000.0]), (C, 1)))
    duh = pin(fl["DUDt"] if fl.get("DUDt") is not None else np.zeros((C, 3)))
    eps_h = torch.zeros(C, dtype=torch.float64).pin_memory()
    us_h = torch.zeros((C, 3), dtype=torch.float64).pin_memory()
    F_h = torch.zeros((C, 3), dtype=torch.float64).pin_memory()
    ge = sedi.Sedi(dict(prm, precision_form="split", use_graphs=1), stream=stream)
    ge.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])

    def step():
        ge.set_fluid(U=Uh.numpy(), grad_p=gph.numpy(), DUDt=duh.numpy())
        ge.step(SUBSTEPS)
        ge.average(eps_h.numpy(), us_h.numpy(), F_h.numpy())

    for _ in range(args.settle + args.warmup):
        step()
    torch.cuda.synchronize()
    K2 = max(3, min(args.steps, 10))
    t_start = time.perf_counter()
    for _ in range(K2):
        step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t_start
    ge.close()
    return {"value": round(world * n * SUBSTEPS * K2 / e2e_s, 1), "unit": UNIT,
            "h2d_bytes_per_step": 3 * C * 3 * 8, "d2h_bytes_per_step": 7 * C * 8, "steps": K2}


def plain_form_leg(prm, parts, fl, stream, args):
    """The other arithmetic forms on the same workload and GPU (the precision pattern):
    the plain FP32 form (the comparison baseline; it cannot reach the 1e-5 force
    tolerance) and the FP64 form (the one other form that meets it, i.e. the comparison
    at matched error), each with throughput and its substep roofline; plus, on the
    200,000-sphere bed, each form's force error at one identical state and its position
    error after 100 substeps against the FP64 form (which matches the oracle to 1e-12)."""
    import torch

    n = len(parts["x"])
    out = {}
    for form, steps in (("plain", max(3, args.steps // 2)), ("fp64", 2)):
        gp, mp = measure(prm, parts, fl, form, steps, min(args.warmup, 1), 0 if form == "fp64" else args.settle,
                         stream, profile=1)
        out[form] = {"value": round(n * SUBSTEPS * len(mp["ms"]) / (np.sum(mp["ms"]) / 1e3), 1),
                     "unit": UNIT, "ms_per_step": round(float(np.mean(mp["ms"])), 4),
                     "roofline": roofline(prm, n, gp, mp["substep_launch_ms"],
                                          gp.stats()["substep_variant"], form=form)}
        gp.close()
        del gp
        torch.cuda.empty_cache()
    out["errors_vs_fp64_on_bed200k"] = form_errors(stream)
    return out


def form_errors(stream, substeps=100):
    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import bed_case

    prm, parts, fl = bed_case()
    rng = np.random.default_rng(29)
    n = len(parts["x"])
    parts = dict(parts, v=rng.normal(0, 0.01, (n, 3)), w=rng.normal(0, 20.0, (n, 3)))
    res = {}
    for form in ("fp64", "split", "plain"):
        h = sedi.Sedi(dict(prm, precision_form=form, use_graphs=0), stream=stream)
        h.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        h.set_fluid(U=fl["U"])
        h.average_inplace()
        f = h.compute_forces()
        h.step(substeps)
        res[form] = (f, h.get_particles()[0])
        h.close()
    L = np.array(prm["hi"]) - np.array(prm["lo"])
    out = {}
    for form in ("split", "plain"):
        e = {}
        for k in ("contact", "lub", "fluid", "torque"):
            ref = np.abs(res["fp64"][0][k]).max()
            e[k] = float(f"{np.abs(res[form][0][k] - res['fp64'][0][k]).max() / ref:.3e}")
        dx = res[form][1] - res["fp64"][1]
        dx -= L * np.round(dx / L) * np.array(prm["periodic"])
        e[f"position_after_{substeps}_substeps_over_d"] = float(
            f"{(np.abs(dx).max(axis=1) / parts['d']).max():.3e}")
        out[form] = e
    return out


def bed200k_leg(args):
    """The sheared 200,000-sphere bed (64 x 32 x 64 mm channel, 64 x 32 x 64 mesh):
    throughput with the L2 flushed between steps (the state fits L2), and the
    substep launch's roofline (the case the ncu captures in profiles/ are taken on)."""
    import torch

    from paper_1601_03801_gb300.workloads import bed_case

    prm, parts, fl = bed_case()
    n = len(parts["x"])
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    g, m = measure(prm, parts, fl, "split", max(args.steps, 20), args.warmup, args.settle, stream,
                   flush=flush, profile=1)
    out = {"workload": WORKLOAD_200K, "particles": n,
           "value": round(n * SUBSTEPS * len(m["ms"]) / (np.sum(m["ms"]) / 1e3), 1), "unit": UNIT,
           "ms_per_step": round(float(np.mean(m["ms"])), 4),
           "l2": "flushed (256 MB write) between timed steps, outside the events",
           "phases_ms_per_step": m["phases"],
           "substep_variant": tuned_launch(g.stats()),
           "roofline": roofline(prm, n, g, m["substep_launch_ms"], g.stats()["substep_variant"],
                                traffic=TRAFFIC_200K)}
    g.close()
    return out


def bounce_leg():
    """Case 1 (Sec. 4.1): a 6 mm sphere falls onto the floor through quiescent fluid;
    the effective restitution e = e_water / e_air (e_air = 0.97, the dry coefficient of
    the linear contact law) over Stokes numbers set by density and viscosity, with
    lubrication and added mass and without them.  Qualitative: the paper compares with
    experimental data that are not available here."""
    from paper_1601_03801_gb300 import diagnostics as dg
    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import bounce_case
    d, out = 6e-3, []
    t0 = time.time()
    for rho_p, nu in ((7800, 1e-6), (2500, 1e-6), (7800, 1e-5), (2500, 1e-5), (7800, 3e-5), (7800, 1e-4)):
        dt = dg.linear_contact_time(800.0, rho_p * math.pi / 6 * d ** 3, 0.97) / 50
        row = {"rho_p": rho_p, "nu_f": nu, "dt": dt}
        for key, on in (("e_eff", 1), ("e_eff_without_lub_added_mass", 0)):
            prm, parts = bounce_case(rho_p, nu, dt, d=d, lubrication=on, added_mass=on)
            g = sedi.Sedi(dict(prm, precision_form="split"))
            g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
            v_in, v_out, _ = dg.bounce_velocities(g, chunk=10)
            row[key] = round(v_out / abs(v_in) / 0.97, 4)
            if on:
                row["impact_speed"] = round(-v_in, 4)
                row["St"] = round(dg.stokes_number(rho_p, d, v_in, nu, 1000.0), 1)
        out.append(row)
    return {"workload": "Case 1: 6 mm sphere, 100 x 100 x 500 mm box of quiescent fluid, k_n = 800 N/m, "
                        "e = 0.97, mu = 0.1, dt = t_c / 50", "sweep": out,
            "wall_s": round(time.time() - t0, 2)}


def ensemble_leg(steps=3, warmup=2, settle=11):
    """256 independent beds of 2,000..50,000 spheres (log-uniform) on 16^3..48^3
    meshes: one ensemble handle (one launch per phase over all beds, one CUDA graph
    per fluid step, batched averaging) against the same beds in 256 single-bed
    handles stepped one after the other.  A step = 20 substeps + 1 averaging of
    every bed; particle-steps/s of all beds together.  The ensemble first runs
    `settle` untimed steps, so that its autotuner (after 200 substeps) has picked the
    batched substep's launch shape and the bins per list cutoff of every bed; the
    single-bed handles run their default shape (the per-particle loop, 128 x 6).  A
    second ensemble handle runs the substeps of each step in one persistent
    cooperative launch instead of the graph (same launch shape after tuning, same
    bits: checked on the first and last bed)."""
    import torch

    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import ensemble_case

    prm, beds = ensemble_case()
    n_total = int(sum(len(b["parts"]["x"]) for b in beds))
    stream = torch.cuda.Stream()

    def load(g, b, bd, kw):
        p = bd["parts"]
        g.set_particles(p["x"], p["v"], p["w"], p["d"], p["rho"], **kw)
        g.set_fluid(U=bd["U"], **kw)

    def ensemble(**extra):
        h = sedi.Sedi(dict(prm, n_beds=len(beds), precision_form="split", **extra), stream=stream)
        for b, bd in enumerate(beds):
            h.set_bed(b, bd["lo"], bd["hi"], bd["ncell"])
            load(h, b, bd, {"bed": b})
        return h

    E = ensemble()
    Ep = ensemble(ens_persistent=1)
    singles = []
    for bd in beds:
        g = sedi.Sedi(dict(prm, lo=bd["lo"], hi=bd["hi"], ncell=bd["ncell"], precision_form="split"),
                      stream=stream)
        load(g, 0, bd, {})
        singles.append(g)

    def timed(step):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def step_batched():
        E.step(SUBSTEPS)
        E.average_inplace()

    def step_persistent():
        Ep.step(SUBSTEPS)
        Ep.average_inplace()

    def step_per_bed():
        for g in singles:
            g.step(SUBSTEPS)
            g.average_inplace()

    E.average_inplace()
    Ep.average_inplace()
    for g in singles:
        g.average_inplace()
    for _ in range(settle):
        step_batched()
        step_persistent()
    torch.cuda.synchronize()
    tuned = E.stats()
    ms_b = timed(step_batched)
    ms_q = timed(step_persistent)
    ms_p = timed(step_per_bed)
    same = all(np.array_equal(a, b) for bed in (0, len(beds) - 1)
               for a, b in zip(E.get_particles(bed=bed), Ep.get_particles(bed=bed)))
    rate = lambda ms: round(n_total * SUBSTEPS / (ms / 1e3), 1)
    return {"workload": "256 beds, N_b = exp(U[ln 2000, ln 50000]) spheres of d = 0.5 mm on a jittered "
                        "lattice, n_b mm cubic periodic-x/y wall-z boxes, n_b^3 meshes (n_b = 16..48), "
                        "log-law flow; step = 20 substeps + 1 averaging of every bed",
            "beds": len(beds), "particles": n_total, "steps": steps, "warmup": warmup,
            "batched": {"value": rate(ms_b), "unit": UNIT, "ms_per_step": round(ms_b, 3)},
            "per_bed_launches": {"value": rate(ms_p), "unit": UNIT, "ms_per_step": round(ms_p, 3)},
            "persistent": {"value": rate(ms_q), "unit": UNIT, "ms_per_step": round(ms_q, 3),
                           "structure": "the 20 substeps of a step in one persistent cooperative "
                                        "launch over all beds (bounded grid barrier between "
                                        "substeps; a rebuild ends the launch, the next resumes)",
                           "same_bits_as_graph": bool(same)},
            "speedup": round(ms_p / ms_b, 3),
            "launch_structure": "per fluid step: one CUDA graph of 20 substeps (a conditional "
                                "batched rebuild node, then one batched substep launch over all "
                                "beds, grid.y = bed), then one batched deposition and one "
                                "persistent smoothing launch for all beds",
            "tuned": {"substep_variant": tuned["substep_variant"], "block": tuned["substep_block"],
                      "bins_per_cutoff": tuned["bins_per_cutoff"],
                      "bin_order": "xz"[tuned["bin_order"]] + " fastest", "settle_steps_untimed": settle},
            "timing": "CUDA events on the launching stream around the steps (the averagings "
                      "synchronise the host once per handle per step)"}


def cnn_warm_start(prm0, parts, fl, snapshots=16, held=2, train_steps=(700, 300)):
    """Learned warm start of the smoothing solve on the 128 x 64 x 128 mesh (0.5 mm
    cells) of the 200,000-sphere bed (the network is this project's addition; Sec. 2.4
    solves the diffusion equation directly).  Training pairs (phi^m, phi^{m+1}) of
    (eps_s, F) are made by the method on the GPU: `snapshots` states of a running bed,
    each deposited and smoothed one backward-Euler pseudo-step at a time (4 pairs per
    state); the last `held` states are held out.  The network is trained on the GPU
    (Adam, lr 2e-3 then 5e-4); with the guess every pseudo-step starts from it.
    Reported on the held-out states: solver steps and smoothing time (inference
    included) from phi^m and from the guess, in the split form (FP32 Chebyshev
    recursion with a double-float residual: a guess saves at most a refinement round)
    and in the FP64 form (steps follow the starting residual); and the error of both
    split-form results against the FP64 oracle at a seeded state (the settled bed with
    seeded velocities, not a training state)."""
    import torch

    from oracle import oracle as orc
    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import storage_round

    prm = dict(prm0, ncell=(128, 64, 128))
    n_tau = prm["n_tau"]
    U = _resample_u(fl["U"], prm0["ncell"], prm["ncell"])
    run = sedi.Sedi(dict(prm, precision_form="split"))
    run.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    run.set_fluid(U=U)
    run.average_inplace()
    one = sedi.Sedi(dict(prm, precision_form="split", n_tau=1,
                         bandwidth=tuple(b / np.sqrt(n_tau) for b in prm["bandwidth"])))
    S0, S1 = prm["shift_eps"], prm["shift_force"]
    pairs, states = [], []
    t0 = time.perf_counter()
    for _ in range(snapshots):
        run.step(SUBSTEPS * 2)
        run.average_inplace()
        states.append(run.get_particles()[:3])
        q = run.deposit()
        phi = np.stack([np.ldexp(q[0].astype(float), -S0)] +
                       [np.ldexp(q[4 + a].astype(float), -S1) for a in range(3)]).astype(np.float32)
        for _m in range(n_tau):
            nxt, _ = one.smooth(phi.astype(np.float64))
            nxt = nxt.astype(np.float32)
            pairs.append((phi, nxt))
            phi = nxt
    gen_s = time.perf_counter() - t0
    run.close()
    one.close()
    train = pairs[:-held * n_tau]
    scale = np.maximum(np.abs(np.stack([p[0] for p in train])).max(axis=(0, 2)), 1e-30).astype(np.float64)
    xs = np.stack([p[0] / scale[:, None] for p in train]).astype(np.float64)
    ts = np.stack([(p[1] - p[0]) / scale[:, None] for p in train]).astype(np.float64)
    del pairs
    rng = np.random.default_rng(1601038015)
    params = []
    for li, (ci, co) in enumerate([(4, 32), (32, 32), (32, 4)]):
        w = rng.normal(0, np.sqrt(2.0 / (27 * ci)), co * ci * 27) * (0.0 if li == 2 else 1.0)
        params += [w, np.zeros(co)]
    trainer = sedi.Sedi(dict(prm, precision_form="split"))
    trainer.cnn_set_params(np.concatenate(params))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = np.concatenate([trainer.cnn_train(xs, ts, steps=train_steps[0], lr=2e-3),
                             trainer.cnn_train(xs, ts, steps=train_steps[1], lr=5e-4)])
    train_s = time.perf_counter() - t0
    trained = trainer.cnn_get_params()
    trainer.close()
    del xs, ts

    def averaged(form, warm, state, reps=2):
        h = sedi.Sedi(dict(prm, precision_form=form, use_cnn_guess=warm, cnn_scale=tuple(scale),
                           profile=1))
        h.set_particles(*state, parts["d"], parts["rho"])
        h.set_fluid(U=U)
        h.cnn_set_params(trained)
        h.average_inplace()  # warm-up
        t_a, i_a = h.timings(), h.stats()["cg_iterations"]
        for _ in range(reps):
            h.average_inplace()
        t_b, i_b = h.timings(), h.stats()["cg_iterations"]
        h.close()
        return (i_b - i_a) / reps / 7.0, (t_b["smooth_ms"] - t_a["smooth_ms"]) / reps

    held_out = {}
    for form in ("split", "fp64"):
        r = {0: [0.0, 0.0], 1: [0.0, 0.0]}
        for state in states[-held:]:
            for warm in (0, 1):
                it, ms = averaged(form, warm, state)
                r[warm][0] += it / held
                r[warm][1] += ms / held
        held_out[form] = {"steps_per_field_cold": round(r[0][0], 1), "steps_per_field_warm": round(r[1][0], 1),
                          "smooth_ms_cold": round(r[0][1], 3), "smooth_ms_warm": round(r[1][1], 3)}
    # error against the FP64 oracle at a seeded state that was not trained on
    srng = np.random.default_rng(1601038016)
    n = len(parts["x"])
    seeded = dict(parts, v=srng.normal(0, 0.01, (n, 3)))
    res = {}
    for warm in (0, 1):
        h = sedi.Sedi(dict(prm, precision_form="split", use_cnn_guess=warm, cnn_scale=tuple(scale)))
        h.set_particles(seeded["x"], seeded["v"], seeded["w"], seeded["d"], seeded["rho"])
        h.set_fluid(U=U)
        h.cnn_set_params(trained)
        res[warm] = h.average()
        h.close()
    o = orc.Oracle(prm, threads=host_cores())
    o.set_particles(*(storage_round(seeded[k], "split") for k in ("x", "v", "w")), seeded["d"], seeded["rho"])
    o.set_fluid(U=U)
    eo, _, Fo = o.average()
    err = {}
    for warm, key in ((0, "cold"), (1, "warm")):
        eg, _, Fg = res[warm]
        err[key] = {"eps_s": float(f"{np.abs(eg - eo).max() / np.abs(eo).max():.3e}"),
                    "F_fp": float(f"{np.abs(Fg - Fo).max() / np.abs(Fo).max():.3e}")}
    return {"mesh": list(prm["ncell"]), "train_pairs": len(train), "held_out_pairs": held * n_tau,
            "snapshots": snapshots, "train_steps": int(sum(train_steps)), "pairs_s": round(gen_s, 2),
            "train_s": round(train_s, 2), "loss_first": float(losses[:5].mean()),
            "loss_last": float(losses[-20:].mean()), "held_out": held_out,
            "error_vs_fp64_oracle": err,
            "note": ("steps per field per averaging (4 pseudo-steps, Chebyshev steps plus one "
                     "true residual per refinement round); smooth_ms_warm includes the network "
                     "inference of every pseudo-step")}


def _resample_u(U, nc_from, nc_to):
    """Nearest-cell copy of a cell-centred field onto a finer uniform mesh."""
    nx, ny, nz = nc_from
    f = U.reshape(nz, ny, nx, 3)
    iz = (np.arange(nc_to[2]) * nz) // nc_to[2]
    iy = (np.arange(nc_to[1]) * ny) // nc_to[1]
    ix = (np.arange(nc_to[0]) * nx) // nc_to[0]
    return f[iz][:, iy][:, :, ix].reshape(-1, 3)


def oracle_sample(prm, parts, fl, threads, substeps, with_average=True):
    """Time the FP64 oracle on a bounded sample of the large bed: the 100 x 100 mm
    patch (large_patch: 1/8 of the spheres and cells, the same bed) for `substeps`
    substeps and one averaging, on `threads` host threads.  Returns (spheres,
    seconds per substep, seconds per averaging)."""
    from oracle import oracle as orc
    from paper_1601_03801_gb300.workloads import large_patch

    pprm, pparts, pfl = large_patch(prm, parts, fl)
    o = orc.Oracle(pprm, threads=threads)
    o.set_particles(pparts["x"], pparts["v"], pparts["w"], pparts["d"], pparts["rho"])
    o.set_fluid(U=pfl["U"], DUDt=pfl["DUDt"])
    t0 = time.perf_counter()
    if with_average:
        o.average()
    t_avg = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.step(substeps)
    t_sub = (time.perf_counter() - t0) / substeps
    return len(pparts["x"]), t_sub, t_avg


def cpu_baseline(prm, parts, fl):
    """The FP64 oracle on this host on a bounded sample of the headline workload
    (oracle_sample): all host cores (3 substeps + 1 averaging) and one core (1 substep
    + 1 averaging), each combined as 20 substeps + 1 averaging per step."""
    cores = host_cores()
    n_all, sub_all, avg_all = oracle_sample(prm, parts, fl, cores, 3)
    n_one, sub_one, avg_one = oracle_sample(prm, parts, fl, 1, 1)
    rate = lambda n, sub, avg: round(n * SUBSTEPS / (SUBSTEPS * sub + avg), 1)
    return {"value": rate(n_all, sub_all, avg_all), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"100 x 100 mm patch of the large bed ({n_all} spheres, 64x64x64 cells, the same "
                       f"tiled bed): 3 oracle substeps ({sub_all:.3f} s each) + 1 averaging "
                       f"({avg_all:.3f} s) on {cores} threads, combined as 20 substeps + 1 averaging"),
            "single_core": {"value": rate(n_one, sub_one, avg_one), "cores": 1,
                            "sample": f"same patch: 1 substep ({sub_one:.3f} s) + 1 averaging "
                                      f"({avg_one:.3f} s) on 1 thread"},
            "nproc": os.cpu_count()}


def reference_arm(args):
    """--impl reference: the FP64 oracle as it stands, on this host's cores, with no
    GPU and without the CUDA library.  Each step is a bounded sample of the headline
    workload: one oracle substep of the 100 x 100 mm patch of the large bed (1/8 of it,
    the same tiled bed, oracle_sample), with the averaging after every 20th step, so
    20 steps are one fluid step of the patch."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1601_03801_gb300.workloads import large_case, large_patch

    prm, parts, fl = large_case()
    pprm, pparts, pfl = large_patch(prm, parts, fl)
    n = len(pparts["x"])
    cores = host_cores()
    o = orc.Oracle(pprm, threads=cores)
    o.set_particles(pparts["x"], pparts["v"], pparts["w"], pparts["d"], pparts["rho"])
    o.set_fluid(U=pfl["U"], DUDt=pfl["DUDt"])
    o.average()  # untimed: the drag sees a smoothed solid fraction
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    n_avg = 0
    for s in range(args.steps):
        o.step(1)
        if (s + 1) % SUBSTEPS == 0:
            o.average()
            n_avg += 1
    total = time.perf_counter() - t0
    value = n * args.steps / total
    sample = (f"each step: 1 oracle substep of the 100 x 100 mm patch of the large bed ({n} spheres, "
              f"64x64x64 cells, 1/8 of the bed), averaging after every 20th step ({n_avg} in the "
              f"timed region), {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / max(1, args.steps) * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_gpu": len(parts["x"]),
                       "substeps_per_step": SUBSTEPS, "sample_particles": n,
                       "step": "one substep of the sample; averaging every 20th step"},
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def kernels_only(args):
    """Run a workload for a few steps without timing (profiling driver: the command
    an ncu capture wraps).  --case bed200k (default), large, patch, smooth (the
    smoother alone on the large bed's mesh) or small."""
    import torch

    from paper_1601_03801_gb300 import sedi
    from paper_1601_03801_gb300.workloads import bed_case, default_params, large_case, large_patch, small_case

    torch.cuda.set_device(0)
    if args.case == "large":
        prm, parts, fl = large_case()
    elif args.case == "patch":
        # a 100 x 100 mm patch of the large bed (1.25M spheres, a few GB on the device):
        # the profiling case whose working set is larger than L2
        prm, parts, fl = large_patch(*large_case())
    elif args.case == "smooth":
        # the smoother alone: 7 seeded fields on the large bed's 256 x 128 x 64 mesh
        from paper_1601_03801_gb300.workloads import random_fields
        prm = default_params(hi=(400e-3, 200e-3, 100e-3), ncell=(256, 128, 64), wall_hi=(0, 0, 0),
                             bandwidth=(1.5e-3,) * 3)
        g = sedi.Sedi(dict(prm, precision_form=args.form))
        phi = random_fields(prm["ncell"], 7, 3)
        for _ in range(args.settle + args.steps):
            _, it = g.smooth(phi)
        print(json.dumps({"mode": "kernels", "case": "smooth", "form": args.form,
                          "calls": args.settle + args.steps, "steps_per_field": it.tolist()}))
        return
    elif args.case == "small":
        prm, parts = small_case(parity_addon=True)
        fl = {"U": None}
    else:
        prm, parts, fl = bed_case()
    extra = {}
    if args.with_cnn:
        extra = dict(use_cnn_guess=1, cnn_scale=(0.6, 1e4, 1e4, 1e4))
    g = sedi.Sedi(dict(prm, precision_form=args.form, use_graphs=int(args.graphs),
                       substep_variant=args.variant, bins_per_cutoff=args.bins,
                       bin_order=args.bin_order, **extra))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.set_fluid(U=fl["U"], DUDt=fl.get("DUDt"))
    if args.with_cnn:
        rng = np.random.default_rng(7)
        g.cnn_set_params(rng.normal(0, 0.05, g.CNN_PARAMS))
    g.average_inplace()
    for _ in range(args.settle + args.steps):
        g.step(SUBSTEPS)
        g.average_inplace()
    g.sync()
    print(json.dumps({"mode": "kernels", "case": args.case, "form": args.form,
                      "steps": args.settle + args.steps, "stats": g.stats()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 20 fluid steps of the 10M bed: a few seconds of timed work, several clock samples
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-cnn", action="store_true", help="skip the learned-warm-start leg")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 256-bed ensemble leg")
    ap.add_argument("--no-bed200k", action="store_true", help="skip the 200,000-sphere leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 form leg")
    ap.add_argument("--no-bounce", action="store_true", help="skip the Case-1 bounce sweep")
    ap.add_argument("--settle", type=int, default=10,
                    help="untimed steps before the warm-up (the method settles the bed further)")
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels"],
                    help="kernels: run a workload untimed (profiling driver)")
    ap.add_argument("--case", default="bed200k", choices=["bed200k", "large", "patch", "smooth", "small"],
                    help="kernels mode: workload")
    ap.add_argument("--form", default="split", choices=["split", "plain", "fp64"])
    ap.add_argument("--with-cnn", action="store_true",
                    help="kernels mode: average with the learned warm start (random weights)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="kernels mode: substep launch variant (-1: autotuned)")
    ap.add_argument("--graphs", type=int, default=1,
                    help="kernels mode: 0 launches kernels one by one (profilers see them)")
    ap.add_argument("--bins", type=int, default=0,
                    help="kernels mode: bins per list cutoff (0: the library's choice)")
    ap.add_argument("--bin-order", type=int, default=-1,
                    help="kernels mode: bin storage order, 0 x fastest, 1 z fastest (-1: the library's choice)")
    args = ap.parse_args()
    if args.mode == "kernels":
        kernels_only(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
