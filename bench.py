#!/usr/bin/env python
"""Throughput benchmark of the DEM hot path on the paper-scale bed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload (the 34M-sphere configuration): 11,000,000 clumps of 1-6 spheres
(~34M spheres, radii lognormal median 2 mm), 4 materials, a 4 x 2 m box with a
plate sliding at 0.2 m/s on top, FP32 forces with voxel positions, dt 1e-6 s,
plain fixed margin (the enlarged-geometry list of section 2.2, rebuilt every K
steps).  The bed is prepared by settling a patch and copy-pasting it (section
4.1).  Metric: sphere-steps per second (and listed contacts per second).

N > 1 (torchrun): every rank runs its own replica (the method does not shard
a scene without a halo exchange); value = all ranks' sphere-steps / max time.
--impl reference: the FP64 CPU oracle, on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sphere-steps/sec and contacts/sec at 1 GB300 (plain vs learned-margin/batched)"
UNIT = "sphere-steps/s"
MARGIN_VBOUND = 1.0   # m/s speed bound behind the fixed margin
K_REBUILD = 20        # steps between list rebuilds
N_CLUMPS_FULL = 11_000_000  # the paper-scale bed


# ---------------------------------------------------------------------------
# roofline bytes
# ---------------------------------------------------------------------------
# The method's algorithmic bytes per force step (FP32 voxel mode), the minimum
# any implementation moves: per listed contact its pair ids (8 B) and FP64
# tangential history read + write (48 B); per sphere its owner and component
# id (8 B); per clump the pose and velocity read for the forces (64 B) and
# the force/torque accumulation (24 B), and for the integration the force and
# torque read (24 B), FP64 velocity and angular velocity read + write (96 B),
# position read + write (48 B), orientation read + write (32 B) and FP32
# mirrors written (40 B).  The update kernel is charged the integration part
# (240 B per clump) and the sphere ids; the pair kernel the contacts, the
# sphere ids and the force part (88 B per clump).
def ALGO_UPDATE(ncl, ns):
    return 240 * ncl + 8 * ns


def ALGO_PAIRS(ncl, ns, n_pairs):
    return 56 * n_pairs + 8 * ns + 88 * ncl


# This implementation's own bytes per launch.  Update: per clump 156 B read
# (force and torque 32, template and scene 8, voxel 16, offset 16,
# orientation 32, velocity record 48, first-sphere index 4; the 48-byte
# certificate reference only for the clumps whose motion bound reaches their
# margin, none in this workload) and 160 B written (offset, orientation,
# velocity record, FP32 mirrors 32, cleared accumulators 32; the voxel only
# when it changes); per sphere its 16-byte pose record written.
# Pair forces: per listed pair its ids (8 B) and its record (20 B: both
# sides' owner and radius and the pair-material row, written at the
# rebuild); per active
# contact the history read + write (48 B); per sphere its pose record (16 B)
# read once; per clump voxel and offset (32 B), velocity mirrors (32 B) and
# accumulators read + written (64 B).
def IMPL_UPDATE(ncl, ns):
    return 316 * ncl + 16 * ns


def IMPL_PAIRS(ncl, ns, n_pairs, n_active):
    return 28 * n_pairs + 48 * n_active + 16 * ns + 128 * ncl


# DRAM bytes (read + write) of one launch in an ncu capture of the same
# kernel on the 687,504-clump bed of the same depth (--footprint 1x0.5), with
# that launch's algorithmic bytes; a launch on a bed of this family is scaled
# by its algorithmic bytes (both grow with the clumps, spheres and pairs in
# the same proportions).  None once the kernel changes.
TRAFFIC = {"k_update32": (140.305664e6 + 87.813376e6, 181879360),
           "k_pairs32": (216.608256e6 + 41.233920e6, 202121440)}
TRAFFIC_SRC = {k: "ncu dram__bytes_read.sum + dram__bytes_write.sum, 687,504-clump bed, scaled "
                  "by algorithmic bytes (profiles/ncu_pairs_update_bed_2M_spheres.md)"
               for k in TRAFFIC}


def roof(kernel, ms, algo, impl, peak, peak_src, full_bed):
    achieved = algo / (ms / 1000.0) / 1e9
    tr = None
    if full_bed and TRAFFIC[kernel] is not None:
        meas, algo_meas = TRAFFIC[kernel]
        tr = meas * algo / algo_meas
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": tr,
            "traffic_source": TRAFFIC_SRC[kernel] if tr is not None else None,
            "kernel": kernel, "kernel_ms": ms, "algorithmic_bytes": algo,
            "impl_bytes": impl, "impl_frac": impl / (ms / 1000.0) / 1e9 / peak,
            "peak_source": peak_src}


def workload_name(n_clumps, n_spheres):
    sph = f"{n_spheres:,}" if n_spheres else "~34,000,000"
    return (f"paper-scale bed: {n_clumps:,} clumps / {sph} spheres, 30 templates of 1-6 "
            "spheres, 4 materials, 4x2 m box, plate sliding 0.2 m/s, FP32 forces + voxel "
            "positions, plain fixed margin")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 100 ms.  Started before the last untimed steps
    (its start-up would otherwise overlap the first milliseconds of the timed
    region); mark_start() / mark_end() bracket the timed region, and the
    summary keeps the samples taken inside it (else those within 0.25 s of
    it, else all)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def _samples(self):
        import datetime

        out = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                out.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        return out

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        allx = self._samples()
        window, pick = "all samples", allx
        if self.t0 is not None and self.t1 is not None:
            inside = [s for s in allx if self.t0 <= s[0] <= self.t1]
            near = [s for s in allx if self.t0 - 0.25 <= s[0] <= self.t1 + 0.25]
            if inside:
                window, pick = "timed region", inside
            elif near:
                window, pick = "within 0.25 s of the timed region", near
        if not pick:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = {nm for s in pick for nm, v in zip(names, s[3]) if v.lower() == "active"}
        return {"sm_mhz": float(np.median([s[1] for s in pick])),
                "sm_max_mhz": float(max(s[2] for s in pick)), "reasons": sorted(reasons),
                "samples": len(pick), "window": window}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample_scene(n_clumps=1500, seed=1239):
    """Clumps of the workload (same templates, materials, dt) in a small box,
    on a lattice squeezed to 0.88 of the mean bounding diameter, which lists
    about as many pairs per sphere (~1.1) as the settled bed does."""
    from paper_2307_03445_gb300 import scenes

    base = scenes.config5(seed=seed, n_clumps=1)
    rng = np.random.default_rng(seed + 7)
    tpl = rng.integers(0, len(base.tpl_mass), size=n_clumps).astype(np.int32)
    bound = base.bounding_radius()[tpl]
    spacing = 0.88 * 2.0 * float(np.mean(bound))
    side = spacing * math.ceil((n_clumps / 2.0) ** 0.5)
    P = scenes.lattice_positions(n_clumps, spacing, 0.0, side, 0.0, side, 0.0, rng, 0.1 * spacing)
    P[:, 2] += float(bound.max())
    base.tpl, base.pos = tpl, P
    base.quat = scenes.random_quaternions(rng, n_clumps)
    base.vel = rng.normal(scale=0.01, size=(n_clumps, 3))
    base.angvel = np.zeros((n_clumps, 3))
    base.walls = scenes.box_walls(-0.01, side + 0.01, -0.01, side + 0.01, 0.0)
    base.lo = (-0.02, -0.02, -0.01)
    base.hi = (side + 0.02, side + 0.02, float(P[:, 2].max()) + 0.02)
    return base


ORACLE_WINDOW = 5 * K_REBUILD  # steps per window of the oracle sample


def time_oracle(budget_s=15.0, n_clumps=1500, max_steps=None):
    """Times the FP64 CPU oracle on the sample scene in windows of
    ORACLE_WINDOW steps (rebuild every K_REBUILD), each from the generated
    state: over thousands of steps the squeezed lattice would fly apart and
    list far fewer pairs than the bed.  Stops after `budget_s` seconds of
    stepping or `max_steps` steps.  Set-up of each window is not timed."""
    import oracle

    sc = oracle_sample_scene(n_clumps)
    margin = MARGIN_VBOUND * sc.h * K_REBUILD
    sc.bin_size = 2.0 * (float(sc.tpl_rad.max()) + margin)
    ns = sc.n_spheres
    steps, busy, pairs = 0, 0.0, []
    while busy < budget_s and (max_steps is None or steps < max_steps):
        w = ORACLE_WINDOW if max_steps is None else min(ORACLE_WINDOW, max_steps - steps)
        sim = oracle.OracleSim(sc, margin, K_REBUILD)
        t0 = time.perf_counter()
        sim.step(w)
        busy += time.perf_counter() - t0
        pairs.append(len(sim.contacts()[0]))
        sim.close()
        steps += w
    return {"value": ns * steps / busy, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{n_clumps} clumps / {ns} spheres of the workload's templates and "
                       f"materials, packed in a small box; {steps} steps in windows of "
                       f"{ORACLE_WINDOW} from the generated state, rebuild every {K_REBUILD}; "
                       f"{int(np.mean(pairs))} listed pairs at window ends; "
                       "single-threaded FP64 C"),
            "seconds": busy, "steps": steps, "ms_per_step": 1000.0 * busy / max(1, steps)}


def _oracle_worker(args):
    """One process of the all-cores oracle timing (spawned, so it shares no
    state with a CUDA context of the parent)."""
    budget_s, n_clumps, max_steps, warm = args
    if warm:
        time_oracle(1e9, n_clumps=n_clumps, max_steps=warm)
    return time_oracle(budget_s, n_clumps=n_clumps, max_steps=max_steps)


def time_oracle_all_cores(budget_s=15.0, n_clumps=1500, max_steps=None, warm=0, procs=None):
    """The oracle on every host core: one independent copy of the sample per
    process (the oracle is single-threaded), all running at once.  The rate
    is the sum of the processes' own rates (sphere-steps over each one's
    stepping time); the wall time of the pool is reported beside it."""
    import multiprocessing as mp

    n = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n) as pool:
        res = pool.map(_oracle_worker, [(budget_s, n_clumps, max_steps, warm)] * n)
    wall = time.perf_counter() - t0
    value = float(sum(r["value"] for r in res))
    steps = res[0]["steps"]
    return {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": res[0]["sample"].replace("single-threaded FP64 C",
                                               f"FP64 C, {n} independent single-threaded "
                                               f"copies at once (one per host core)"),
            "seconds": max(r["seconds"] for r in res), "pool_wall_s": wall, "steps": steps,
            "ms_per_step": max(r["ms_per_step"] for r in res),
            "per_process": [r["value"] for r in res]}


# ---------------------------------------------------------------------------
# replicas: one per rank, no data-path collective
# ---------------------------------------------------------------------------
def max_over_ranks(ms, device):
    """The slowest rank's time (every rank receives it)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, ms):
    """Units all ranks processed per second of the slowest rank's time."""
    return world * units_per_rank * steps / (ms / 1000.0)


# ---------------------------------------------------------------------------
# the learned-margin and batched forms
# ---------------------------------------------------------------------------
LEARN_CAND = [1e-6, 2e-6, 4e-6, 8e-6, 1.6e-5, 3.2e-5]  # candidate margins [m]
BIN_FACTORS = (0.5, 0.7, 1.0, 1.4)  # bin edge / (2 x largest enlarged radius) tried


def _timed_steps(sim, stream, n):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def learned_form(dem, sim, stream, steps, ns, plain_st, plain_ms_step, log, start_state=None,
                 intervals=4, interval=80, audited=80, cand=None, safety=2.0, speed_floor=0.0):
    """The learned rebuild rule on the same bed: traces of the plain rule and
    training on the GPU (untimed), then `intervals` whole intervals of
    `interval` steps timed with the learned rule and, from the same state,
    the same number of steps with the plain rule (halt mode: a failed
    certificate ends an interval early).  Then `audited` more learned steps,
    each followed by the exact check against a fresh zero-margin detection
    (missed contacts summed over all of them)."""
    t0 = time.time()
    if start_state is None:
        start_state = sim.state()
    cand = LEARN_CAND if cand is None else cand
    x, t = sim.trace(2, 240, cand, cap=1 << 24)
    reg = dem.Regressor(device=sim_device(sim))
    loss = reg.train(x, t, steps=800, batch=8192, lr=2e-3, seed=1)
    log(f"learned form: {len(x)} trace samples, loss {loss:.4f}, {time.time() - t0:.1f} s")
    n = intervals * interval
    sim.set_timing(True)  # events only: the steps are not serialised
    # the plain rule from the start state over the same steps
    sim.set_state(*start_state)
    sim.reset_stats()
    ms_plain = _timed_steps(sim, stream, n)
    st_plain = sim.stats()
    # the learned rule from the same state; interval x safety stays inside
    # the traced window, where lifetimes are not capped
    sim.set_state(*start_state)
    sim.set_learned_policy(reg, interval=interval, safety=safety, candidates=cand,
                           speed_floor=speed_floor)
    sim.reset_stats()
    ms = _timed_steps(sim, stream, n)
    st = sim.stats()
    sim.set_timing(False)
    missed = 0
    for _ in range(audited):
        sim.step(1)
        missed += sim.audit()
    sim.set_learned_policy(None)
    reg.close()
    return {"value": ns * n / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / n,
            "steps": n, "intervals": intervals, "plain_ms_per_step_same_steps": ms_plain / n,
            "vs_plain": ms_plain / ms,
            # against the headline run's step (the plain rule on the two-level list)
            "vs_headline_step": plain_ms_step / (ms / n), "rebuilds": st["rebuilds"],
            "early_rebuilds": st["early_rebuilds"], "rollbacks": st["rollbacks"],
            "listed_per_step": st["pair_steps"] / max(1, st["steps"]),
            "listed_per_step_plain": st_plain["pair_steps"] / max(1, st_plain["steps"]),
            "rebuilds_plain": st_plain["rebuilds"],
            "missed_contacts": missed, "audited_steps": audited,
            "ms_predict_per_interval": st["ms_predict"] / max(1, st["rebuilds"]),
            "ms_rebuild_per_interval": st["ms_detect"] / max(1, st["rebuilds"]),
            "rule": f"6->3x64->1 MLP (BF16 weights) per bin, candidates {cand[0] * 1e6:g}-"
                    f"{cand[-1] * 1e6:g} um, target "
                    f"interval {interval} x {safety:g}, "
                    + (f"margins at least {speed_floor:g} x h x interval x speed per clump, "
                       if speed_floor > 0 else "")
                    + f"halt on certificate; trained on 2 x 240-step "
                    f"traces; timed over {intervals} whole intervals; exact audit after each of "
                    f"{audited} further steps"}


def outer_form(sim, stream, ns, log, factor=4.0, n_inner=10, cycles=2):
    """The two-level contact list on the same bed: an outer list at factor x
    the margin serves n_inner rebuilds (each a filter of the outer list that
    gives the fresh detection's list).  Timed over whole outer cycles
    (cycles x n_inner x K steps), against the plain rule over the same steps
    from the same state; both with per-phase events."""
    s0 = sim.state()
    n = cycles * n_inner * K_REBUILD
    sim.set_outer_list(factor, 0)  # the plain rule: a fresh detection at every rebuild
    sim.set_timing(True)
    sim.set_state(*s0)
    sim.reset_stats()
    ms_plain = _timed_steps(sim, stream, n)
    st_plain = sim.stats()
    sim.set_state(*s0)
    sim.set_outer_list(factor, n_inner)
    sim.step(n_inner * K_REBUILD)  # the first outer list
    sim.set_state(*s0)
    sim.reset_stats()
    ms = _timed_steps(sim, stream, n)
    st = sim.stats()
    sim.set_outer_list(factor, 0)
    sim.set_timing(False)
    # the same steps without per-phase events (graph-captured steps): plain,
    # outer list, and outer list detected on a second stream while the
    # interval's steps run
    whole = {}
    for name, args in (("plain", (factor, 0)), ("outer", (factor, n_inner)),
                       ("outer_async", (factor, n_inner, True))):
        sim.set_outer_list(*args)
        sim.set_state(*s0)
        sim.step(n_inner * K_REBUILD)  # the first outer list (and the first started on st2)
        sim.set_state(*s0)
        sim.reset_stats()
        whole[name] = _timed_steps(sim, stream, n) / n
        whole[name + "_outer_rebuilds"] = sim.stats()["outer_rebuilds"]
    sim.set_outer_list(factor, 0)
    log(f"outer list: {ms / n:.4f} ms/step vs plain {ms_plain / n:.4f} (per-phase events); "
        f"without events plain {whole['plain']:.4f}, outer {whole['outer']:.4f}, "
        f"outer on a second stream {whole['outer_async']:.4f}")
    return {"value": ns * n / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / n, "steps": n,
            "plain_ms_per_step_same_steps": ms_plain / n, "vs_plain": ms_plain / ms,
            "rebuilds": st["rebuilds"], "outer_rebuilds": st["outer_rebuilds"],
            "rebuild_ms_per_rebuild": st["ms_detect"] / max(1, st["rebuilds"]),
            "plain_rebuild_ms_per_rebuild": st_plain["ms_detect"] / max(1, st_plain["rebuilds"]),
            "ms_per_step_without_phase_events": whole,
            "rule": f"outer list at {factor} x the margin serving {n_inner} rebuilds of the "
                    f"plain rule (each list exactly the fresh detection's); timed over {cycles} "
                    f"whole outer cycles; outer_async: the next outer list detected on a second "
                    f"stream during the interval before it is needed"}


def sim_device(sim):
    import torch

    return torch.cuda.current_device()


def batched_form(dem, steps, device, log, warmup=K_REBUILD):
    """The batched sweep (64 box-settling scenes of 5,000-100,000 clumps, own
    friction and templates): one context with graph-captured steps against
    the same scenes run one context after another."""
    import torch

    from paper_2307_03445_gb300 import scenes

    t0 = time.time()
    parts = scenes.config4()
    first, rest = scenes.merge_batch(parts)
    ns = sum(p.n_spheres for p in parts)
    log(f"batched form: {len(parts)} scenes, {ns} spheres, generated in {time.time() - t0:.1f} s")
    margin = MARGIN_VBOUND * first.h * K_REBUILD
    stream = torch.cuda.Stream()
    sim = dem.Simulation(first, margin=margin, rebuild_interval=K_REBUILD,
                         precision=dem.DEM_FP32_VOXEL, device=device, stream=stream.cuda_stream,
                         extra_scenes=rest)
    sim.set_graphs(True)
    sim.step(warmup)
    fb, _ = sim.autotune_bins(BIN_FACTORS, reps=1)
    tiles = sim.autotune_tiles(steps=6, reps=1)
    sim.step(warmup)
    sim.reset_stats()
    ms_b = _timed_steps(sim, stream, steps)
    launches = sim.stats()["launches"]
    sim.close()
    ms_s = 0.0
    for p in parts:
        one = dem.Simulation(p, margin=margin, rebuild_interval=K_REBUILD,
                             precision=dem.DEM_FP32_VOXEL, device=device, stream=stream.cuda_stream)
        one.set_graphs(True)
        one.step(K_REBUILD)
        one.autotune_bins(BIN_FACTORS, reps=1)
        one.autotune_tiles(steps=6, reps=1)
        one.step(K_REBUILD)
        ms_s += _timed_steps(one, stream, steps)
        one.close()
    return {"value": ns * steps / (ms_b / 1000.0), "unit": UNIT, "ms_per_step": ms_b / steps,
            "per_scene_value": ns * steps / (ms_s / 1000.0),
            "vs_per_scene": ms_s / ms_b, "n_scenes": len(parts), "n_spheres": ns,
            "bin_factor": fb, "tiles": tiles, "launches": launches,
            "workload": "64 box-settling scenes, 5,000-100,000 clumps (log-uniform), own mu "
                        "0.2-0.9 and 10 templates of 1-5 spheres each, FP32 voxel, one context "
                        "with graph-captured steps vs one context per scene"}


# ---------------------------------------------------------------------------
# the other workload shapes (--config 1-4)
# ---------------------------------------------------------------------------
def config_scene(cfg, n_clumps, log):
    """(scene, precision, workload name) of workload shape 1, 2 or 3."""
    from paper_2307_03445_gb300 import scenes, workloads

    if cfg == 1:
        sc = scenes.config1()
        # 0.1 s of the settling first (untimed): the lower layers have landed
        # and the upper ones are still falling onto them
        sc.pos, sc.quat, sc.vel, sc.angvel = workloads.settle(sc, 0.1, log=log)
        name = ("1,000 clumps of 3 overlapping spheres (r 1-2 mm), 1 material, FP64, settling "
                "in a 5x5x10 cm box of planes from a jittered lattice, dt 1e-6 s, timed from "
                "0.1 s into the settling")
        return sc, scenes.PREC_FP64, name
    if cfg == 2:
        base = scenes.config2()
        n = n_clumps or base.n_clumps
        sc = workloads.settled_bed(base, n, 0.0, 0.25, 0.0, 0.25, seed=base.seed, log=log)
        name = (f"{n:,} clumps from 20 templates of 1-5 spheres (r lognormal median 1.5 mm), "
                "4 per-sphere materials, settled in a 0.25 m box, FP32 forces + voxel positions")
        return sc, scenes.PREC_FP32, name
    base = scenes.config3()
    n = n_clumps or 1_000_000
    R = 0.2

    def inside(x, y, b):
        return np.hypot(x, y) <= R - b

    sc = workloads.settled_bed(base, n, -R, R, -R, R, seed=base.seed, inside=inside, log=log)
    # the cone: tip 1 mm above the bed's top at the axis, pushed down at 1 cm/s
    top = float((sc.pos[:, 2] + sc.bounding_radius()[sc.tpl]).max())
    cone = dict(base.cone)
    cone["p"] = (0.0, 0.0, top + 1e-3)
    sc.walls = list(sc.walls) + [cone]
    sc.hi = (sc.hi[0], sc.hi[1], top + 0.1)
    name = (f"{n:,} clumps of 3 spheres (r 1-2 mm) settled in a cylinder of radius 0.2 m, an "
            "analytic cone (30 deg half angle, 2 cm base) pushed down at 1 cm/s, FP32 forces + "
            "FP64 integration")
    return sc, scenes.PREC_FP32, name


def small_config_line(args, dem, workloads, world, rank, local, log):
    """The bench line of workload shape 1, 2, 3 (one scene) or 4 (batched).
    The value is taken with graph-launched steps (these scenes are small
    enough for launch overhead to matter); the per-kernel times come from a
    second, event-timed pass of the same length."""
    import torch

    if args.config == 4:
        b = batched_form(dem, args.steps, local, log, warmup=args.warmup)
        return {"metric": METRIC, "value": world * b["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": b["workload"], "n_spheres": b["n_spheres"],
                           "parallelism": f"replicas{world}",
                           "l2": "inputs larger than L2 (6M spheres)"},
                "forms": {"batched": b}, "gpu_launches": b["launches"], "e2e": None}
    t0 = time.time()
    sc, prec, name = config_scene(args.config, None if args.n_clumps == N_CLUMPS_FULL
                                  else args.n_clumps, log)
    log(f"config {args.config} ready in {time.time() - t0:.1f} s: {sc.n_clumps} clumps, "
        f"{sc.n_spheres} spheres")
    stream = torch.cuda.Stream()
    margin = MARGIN_VBOUND * sc.h * K_REBUILD
    sim = dem.Simulation(sc, margin=margin, rebuild_interval=K_REBUILD, precision=prec,
                         device=local, stream=stream.cuda_stream)
    ns, ncl = sc.n_spheres, sc.n_clumps
    sim.set_graphs(True)
    sim.step(args.warmup)
    if ncl >= 100_000:
        sim.autotune_bins(BIN_FACTORS, reps=1)
        sim.autotune_tiles(steps=6, reps=1)
    with ClockSampler(local) as clk:
        if ncl >= 100_000:
            sim.step(args.warmup)
        s0 = sim.state()
        sim.reset_stats()
        clk.mark_start()
        ms = _timed_steps(sim, stream, args.steps)
        clk.mark_end()
    st = sim.stats()
    if world > 1:
        ms = max_over_ranks(ms, torch.device("cuda", local))
    # the same steps again from the same state with per-kernel events
    sim.set_state(*s0)
    sim.reset_stats()
    sim.set_timing(True)
    _timed_steps(sim, stream, args.steps)
    sim.set_timing(False)
    st2 = sim.stats()
    k = max(1, st2["timed_steps"])
    line = {"metric": METRIC, "value": whole_job_rate(world, ns, args.steps, ms), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
            "contacts_per_sec": whole_job_rate(world, st["pair_steps"], 1, ms),
            "config": {"workload": name, "n_clumps": ncl, "n_spheres": ns,
                       "listed_pairs": st["n_pairs"], "active_contacts": st["active_last"],
                       "wall_contacts": st["n_wall_contacts"], "margin_m": margin,
                       "rebuild_interval": K_REBUILD, "dt": sc.h, "rebuilds": st["rebuilds"],
                       "guard_violations": st["guard_violations"],
                       "parallelism": f"replicas{world}", "launch": "CUDA graphs",
                       "l2": "state smaller than L2 (no flush)" if ns < 1_000_000
                             else "inputs larger than L2",
                       "phase_ms_event_timed_pass": {
                           "pairs": st2["ms_pairs"] / k, "walls": st2["ms_walls"] / k,
                           "update": st2["ms_update"] / k, "rebuild_total": st2["ms_detect"]}},
            "gpu_launches": st["launches"], "clocks": clk.summary(), "e2e": None}
    if not args.no_e2e:
        sim.set_state(*s0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sim.set_state(*s0)
        sim.step(args.steps)
        out = sim.state()
        e2e_ms = (time.perf_counter() - t1) * 1000.0
        if world > 1:
            e2e_ms = max_over_ranks(e2e_ms, torch.device("cuda", local))
        b = ncl * 13 * 8
        line["e2e"] = {"value": whole_job_rate(world, ns, args.steps, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": b / args.steps, "d2h_bytes_per_step": b / args.steps,
                       "steps": args.steps, "host_buffers": "pageable numpy"}
        del out
    if args.config == 3 and not args.no_forms:
        sim.set_state(*s0)
        # the settled cylinder still holds rattling clumps: candidates up to
        # 128 um so that their bins can be given a margin for a whole interval
        line["forms"] = {"learned": learned_form(dem, sim, stream, args.steps, ns, st,
                                                 ms / args.steps, log, start_state=s0,
                                                 cand=LEARN_CAND + [6.4e-5, 1.28e-4],
                                                 speed_floor=1.5)}
    sim.close()
    if rank == 0 and not args.no_cpu_baseline and args.config == 1:
        # the oracle runs this workload whole (1,000 clumps), on one core and on all
        line["cpu_baseline"] = time_oracle_config1(sc, margin, args.steps)
    return line


def time_oracle_config1(sc, margin, steps):
    """The FP64 oracle on the 1,000-clump workload itself, `steps` steps from
    the generated state, single-threaded (its CPU baseline)."""
    import oracle

    sc.bin_size = 2.0 * (float(sc.tpl_rad.max()) + margin)
    sim = oracle.OracleSim(sc, margin, K_REBUILD)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    sim.close()
    return {"value": sc.n_spheres * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the whole workload ({sc.n_clumps} clumps / {sc.n_spheres} spheres), "
                      f"{steps} steps from the same state as the GPU's, single-threaded FP64 C"}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n-clumps", type=int, default=N_CLUMPS_FULL)
    ap.add_argument("--footprint", default="4x2",
                    help="box footprint LXxLY in metres of the paper-scale bed; with the same "
                         "0.25 m patch a smaller footprint gives a bed of the same depth and "
                         "packing with fewer clumps (e.g. 1x0.5 and --n-clumps 687504)")
    ap.add_argument("--oracle-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--boundary", default="analytic", choices=["analytic", "mesh"],
                    help="the box and plate as analytic planes, or as 12 mesh facets with a "
                         "cone of 544 facets pushed into the bed")
    ap.add_argument("--outer-factor", type=float, default=4.0,
                    help="the outer list's margin over the plain margin")
    ap.add_argument("--outer-list", type=int, default=10,
                    help="rebuilds one outer list serves in the timed run; every "
                         "list filtered from it is exactly the fresh detection's (0: every "
                         "rebuild detects afresh)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the learned-margin and batched forms")
    ap.add_argument("--config", type=int, default=5, choices=[1, 2, 3, 4, 5],
                    help="workload: 5 the paper-scale bed (default); 1 the 1,000-clump FP64 "
                         "settling box; 2 the 200,000-clump box; 3 the 1,000,000-clump cylinder "
                         "with a cone, learned vs fixed margin; 4 the batched 64-scene sweep")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # each step: one oracle step over a 20,000-clump sample of the
        # workload, in one independent copy per host core
        cb = time_oracle_all_cores(1e9, n_clumps=20000, max_steps=args.steps, warm=args.warmup)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": cb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.n_clumps, 0) + " (CPU oracle sample)",
                           "sample": cb["sample"]},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    import paper_2307_03445_gb300 as dem
    from paper_2307_03445_gb300 import workloads

    log = (lambda m: print(f"[bench r{rank}] {m}", file=sys.stderr, flush=True))
    if args.config != 5:
        line = small_config_line(args, dem, workloads, world, rank, local, log)
        if rank == 0:
            print(json.dumps(line))
        return
    t0 = time.time()
    lx, ly = (float(v) for v in args.footprint.lower().split("x"))
    sc = workloads.bed_c5(n_clumps=args.n_clumps, lx=lx, ly=ly, log=log)
    if args.boundary == "mesh":
        # the box and sliding plate as 12 facets, and a cone of 544 facets
        # pushed into the bed at 1 cm/s (section 4's cone penetration)
        sc.walls = workloads.facet_box(sc.walls)
        sc = workloads.insert_cone_mesh(sc)
    log(f"bed ready in {time.time() - t0:.1f} s: {sc.n_clumps} clumps, {sc.n_spheres} spheres")
    stream = torch.cuda.Stream()
    margin = MARGIN_VBOUND * sc.h * K_REBUILD
    sim = dem.Simulation(sc, margin=margin, rebuild_interval=K_REBUILD,
                         precision=dem.DEM_FP32_VOXEL, device=local, stream=stream.cuda_stream)
    ns, ncl = sc.n_spheres, sc.n_clumps
    if args.outer_list > 0:
        sim.set_outer_list(args.outer_factor, args.outer_list)
    sim.step(args.warmup)
    bin_factor, bin_ms = sim.autotune_bins(BIN_FACTORS, reps=1)
    log(f"bin autotune: factor {bin_factor} ({bin_ms})")
    tiles = sim.autotune_tiles(steps=6, reps=2)
    log(f"tile autotune: {tiles}")
    sim.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        sim.step(args.warmup)
        sim.reset_stats()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        torch.cuda.nvtx.range_push("timed")  # profilers select the timed launches by this range
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clk.mark_end()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    st = sim.stats()
    if world > 1:
        ms = max_over_ranks(ms, torch.device("cuda", local))
    ms_step = ms / args.steps
    value = whole_job_rate(world, ns, args.steps, ms)
    contacts_ps = whole_job_rate(world, st["pair_steps"], 1, ms)

    # rooflines of the two step kernels against the measured copy bandwidth
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured (burst copy)" if "hbm_gbs" in peaks else "fallback"
    n_pairs, n_active = st["n_pairs"], st["active_last"]
    pair_ms = st["ms_pairs"] / max(1, st["timed_steps"])
    upd_ms = st["ms_update"] / max(1, st["timed_steps"])
    bed_family = args.boundary == "analytic"  # the beds the traffic capture scales to
    rooflines = {
        "k_update32": roof("k_update32", upd_ms, algo=ALGO_UPDATE(ncl, ns),
                           impl=IMPL_UPDATE(ncl, ns), peak=peak, peak_src=peak_src,
                           full_bed=bed_family),
        "k_pairs32": roof("k_pairs32", pair_ms, algo=ALGO_PAIRS(ncl, ns, n_pairs),
                          impl=IMPL_PAIRS(ncl, ns, n_pairs, n_active), peak=peak,
                          peak_src=peak_src, full_bed=bed_family),
    }
    # `roofline` is the kernel with the larger share of the step
    roofline = max(rooflines.values(), key=lambda r: r["kernel_ms"])

    e2e = None
    if not args.no_e2e:
        # inputs and results in pinned host memory (page-locked, so the copies
        # are DMA transfers); the timed region holds the upload, the steps and
        # the read-back
        def pinned(w):
            return torch.empty((ncl, w), dtype=torch.float64, pin_memory=True).numpy()

        inp = [pinned(w) for w in (3, 4, 3, 3)]
        res = [pinned(w) for w in (3, 4, 3, 3)]
        sim.state(out=inp)
        k2 = max(args.steps // 4, K_REBUILD)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sim.set_state(*inp)
        sim.step(k2)
        out = sim.state(out=res)
        t2 = time.perf_counter()
        e2e_ms = (t2 - t1) * 1000.0
        if world > 1:
            e2e_ms = max_over_ranks(e2e_ms, torch.device("cuda", local))
        bytes_state = ncl * 13 * 8
        e2e = {"value": whole_job_rate(world, ns, k2, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": bytes_state / k2, "d2h_bytes_per_step": bytes_state / k2,
               "steps": k2}
        del out
    forms = None
    if not args.no_forms:
        forms = {"outer_list": outer_form(sim, stream, ns, log, factor=args.outer_factor,
                                          n_inner=max(1, args.outer_list)),
                 "learned": learned_form(dem, sim, stream, args.steps, ns, st, ms_step, log,
                                         speed_floor=1.5)}
    sim.close()
    if forms is not None:
        forms["batched"] = batched_form(dem, args.steps, local, log)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        # all host cores (one oracle copy per core), and one core alone
        cb = time_oracle_all_cores(args.oracle_seconds)
        one = time_oracle(args.oracle_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["single_core"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "contacts_per_sec": contacts_ps,
        "config": {"workload": workload_name(ncl, ns) + (
                       " (box and plate as 12 mesh facets, a cone of 544 facets pushed in at "
                       "1 cm/s)" if args.boundary == "mesh" else ""),
                   "boundary": args.boundary, "n_clumps": ncl, "n_spheres": ns,
                   "listed_pairs": n_pairs, "active_contacts": n_active,
                   "wall_contacts": st["n_wall_contacts"], "margin_m": margin,
                   "rebuild_interval": K_REBUILD, "dt": sc.h, "rebuilds": st["rebuilds"],
                   "contact_list": (f"two-level: an outer list at {args.outer_factor:g} x the "
                                    f"margin serves "
                                    f"{args.outer_list} rebuilds, each list filtered from it "
                                    f"with the exact test (equal to a fresh detection); "
                                    f"{st['outer_rebuilds']} outer detections in the timed "
                                    f"steps" if args.outer_list > 0 else
                                    "a fresh detection at every rebuild"),
                   "bin_factor": bin_factor, "bin_autotune_ms": bin_ms, "tiles": tiles,
                   "guard_violations": st["guard_violations"],
                   "l2": "inputs larger than L2 (state ~GBs)", "parallelism": f"replicas{world}",
                   "phase_ms": {"pairs": pair_ms,
                                "walls": st["ms_walls"] / max(1, st["timed_steps"]),
                                "update": st["ms_update"] / max(1, st["timed_steps"]),
                                "rebuild_total": st["ms_detect"]}},
        "forms": forms,
        "roofline": roofline,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": st["launches"],
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
