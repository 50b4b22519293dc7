"""Benchmark of the rail-based KMC sweep on GB300 (site-updates/s).

Workload (N=1): the plain large device -- 65,536 rails x 1,024 sites (64 MiB
uint8 occupancy), 25 % Bernoulli filling, per-site barriers Ea ~ N(0.40, 0.02)
eV, T = 300 K, injecting/extracting electrodes (1e9 Hz), triangular +-2 V sweep
with 1e5 steps per cycle.  One benchmark step = one kmc_step_n call advancing
every rail and site by `--chunk` time steps (default 10,000), so one step is
R * L * chunk site-updates; the default 20 timed steps cover two whole cycles
of the sweep (every phase of the protocol equally), and the end-to-end leg
times the next 20.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kmc|reference]
                    [--scaling weak|strong]

Under torchrun (N > 1) the device is partitioned by rails (rail_base, no
collective on the data path): with --scaling weak (the default) every rank
advances its own 65,536 rails of a device of N x 65,536 rails; with
--scaling strong the ranks split the 65,536 rails.  The timed region is
bracketed by a barrier and the maximum over ranks is reported.
``--impl reference`` times the FP64 CPU oracle on this host's cores on a bounded
sample of the same device (rank 0 only).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_09413_gb300 import workloads as W  # noqa: E402

METRIC = "site-updates/s on 1 GB300 (% HBM roofline)"
UNIT = "site-updates/s"
BYTES_PER_SITE_UPDATE = 2.0        # uint8 read + write per site and step
# IMAD-pipe issue slots per Philox4x32-10 block of one lane whose rail, step and
# instance counter words are warp-uniform: rounds 1 and 2 multiply one per-lane
# word each (the other product is warp-uniform), rounds 3-9 two, round 10 two
# low halves only (its high halves feed words the draw does not use); a
# 32x32->64 widening multiply takes two of the pipe's slots, a low half one:
# 16 x 2 + 2 = 34.
PHILOX_IMAD_SLOTS = 34
IMAD_PER_SM_PER_CLK = 64           # 32-bit integer multiply-add lanes per SM per clock
SMS = 152
SM_MAX_MHZ = 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured", float(d.get("sm_max_mhz", SM_MAX_MHZ))
    except Exception:
        return 6800.0, "fallback", SM_MAX_MHZ


def _traffic_per_launch(rails: int, steps: int):
    """DRAM bytes (read + write) of one sweep launch from the ncu capture in
    profiles/sweep_traffic.json, scaled to `rails` (the per-launch traffic is
    the occupancy and per-site tables, proportional to rails x sites), or None
    when the kernel source changed since the capture or the capture's launch
    covered another number of steps."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["kernel_source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except Exception:
        return None
    if sha != rec.get("kernel_source_sha256") or rec.get("steps_per_launch") != steps:
        return None
    return (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * rails / rec["rails"]


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _voltage(n_needed: int, steps_per_cycle: int = 100000) -> np.ndarray:
    cycles = max(2, -(-n_needed // steps_per_cycle))
    return W.triangle_protocol(2.0, steps_per_cycle, cycles)


def cpu_baseline(wl, budget_s: float, stride: int = 16, steps_per_call: int = 25):
    """Time the FP64 oracle, as it stands, on this host's cores on every
    `stride`-th rail of the device for about `budget_s` seconds."""
    import oracle
    ids = np.arange(0, wl.device.R, stride, dtype=np.int32)
    occ0 = oracle.init_occupancy(wl.device, 1, fill=wl.fill, rail_ids=ids)
    Ea = wl.Ea_site[ids] if wl.Ea_site is not None else None
    sim = oracle.OracleSim(wl.device, wl.V, occ0, Ea, rail_ids=ids)
    t0 = time.perf_counter()
    steps = 0
    while True:
        sim.step_n(steps_per_call)
        steps += steps_per_call
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    su = len(ids) * wl.device.L * steps
    # the same oracle on one core, on every 16th rail of that sample, ~1/4 of the budget
    ids1 = ids[::16]
    n_all = oracle.max_threads()
    occ1 = oracle.init_occupancy(wl.device, 1, fill=wl.fill, rail_ids=ids1)
    Ea1 = wl.Ea_site[ids1] if wl.Ea_site is not None else None
    sim1 = oracle.OracleSim(wl.device, wl.V, occ1, Ea1, rail_ids=ids1, nthreads=1)
    t1 = time.perf_counter()
    steps1 = 0
    while time.perf_counter() - t1 < budget_s / 4:
        sim1.step_n(steps_per_call)
        steps1 += steps_per_call
    el1 = time.perf_counter() - t1
    sim1.nthreads = n_all          # restore the thread count for later oracle calls
    sim1.step_n(0)
    return {"value": su / el, "unit": UNIT, "cores": n_all, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": "%d of %d rails (every %dth) x %d steps of %s, %.1f s" % (
                len(ids), wl.device.R, stride, steps, wl.name, el),
            "one_core": {"value": len(ids1) * wl.device.L * steps1 / el1, "unit": UNIT,
                         "sample": "%d rails x %d steps, %.1f s" % (len(ids1), steps1, el1)}}


def _cpu_model() -> str:
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return ln.split(":", 1)[1].strip()
        with open("/proc/cpuinfo") as f:
            parts = [ln.split(":", 1)[1].strip() for ln in f
                     if ln.split(":")[0].strip() in ("CPU implementer", "CPU part")][:2]
        return "%s (%s)" % (platform.machine(), ", ".join(parts))
    except Exception:
        return platform.machine()


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_needed = (args.warmup + args.steps) * args.ref_steps
    wl = W.hysteresis_65536x1024(R=args.rails, steps_per_cycle=100000, cycles=2)
    wl.V = _voltage(n_needed)
    ids = np.arange(0, wl.device.R, args.ref_stride, dtype=np.int32)
    occ0 = oracle.init_occupancy(wl.device, 1, fill=wl.fill, rail_ids=ids)
    Ea = wl.Ea_site[ids] if wl.Ea_site is not None else None
    sim = oracle.OracleSim(wl.device, wl.V, occ0, Ea, rail_ids=ids)
    for _ in range(args.warmup):
        sim.step_n(args.ref_steps)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sim.step_n(args.ref_steps)
        times.append(time.perf_counter() - t0)
    su_step = len(ids) * wl.device.L * args.ref_steps
    total = sum(times)
    value = su_step * args.steps / total
    sample = "%d of %d rails (every %dth) x %d time steps per step" % (
        len(ids), wl.device.R, args.ref_stride, args.ref_steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "rails": wl.device.R, "sites": wl.device.L,
                   "sample": sample, "parallelism": "OpenMP over rails (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_kmc(args):
    import torch
    from paper_2511_09413_gb300 import kmc
    from paper_2511_09413_gb300 import multigpu as MG

    rank, local_rank, world = _env_rank()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    kmc.load()
    stream = torch.cuda.current_stream()
    chunk = args.chunk
    # rails of this rank: its own 65,536 of a device of world x 65,536 (weak),
    # or its part of the 65,536 (strong); the rail index is global either way
    if args.scaling == "strong":
        r0, r1 = MG.shard_rails(args.rails, rank, world)
    else:
        r0, r1 = rank * args.rails, (rank + 1) * args.rails
    # warm-up, timed and end-to-end steps, and one chunk of slack
    n_needed = (args.warmup + 2 * args.steps + 1) * chunk
    cycles = max(2, -(-n_needed // 100000))
    wl = W.hysteresis_65536x1024(R=r1 - r0, rail_base=r0, steps_per_cycle=100000, cycles=cycles)
    sim = kmc.Sim.from_workload(wl, stream=stream.cuda_stream)
    R, L = wl.device.R, wl.device.L
    su_per_step = R * L * chunk
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        sim.step_n(chunk)
    torch.cuda.synchronize()
    cnt0 = sim.counters()
    t_first = sim.t

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    MG.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush_buf.zero_()                         # evict L2 between timed steps
        ev[i][0].record(stream)
        sim.step_n(chunk)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    MG.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    t_last = sim.t
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_rank = sum(ms_steps)
    cnt1 = sim.counters()
    ms = MG.max_over_ranks(ms_rank, device="cuda")
    # site-updates of every rank in the timed region
    if args.scaling == "strong":
        units = [float((b - a) * L * chunk * args.steps)
                 for a, b in (MG.shard_rails(args.rails, k, world) for k in range(world))]
    else:
        units = [float(args.rails * L * chunk * args.steps)] * world
    value = MG.whole_job_rate(units, ms / 1e3)

    # end to end through the C ABI with host buffers, over as many steps as
    # the timed region: the step's voltage chunk in, its traces out
    from paper_2511_09413_gb300.kmc import kmc_observables, kmc_set_voltage
    Vpin = torch.empty(chunk, dtype=torch.float64, pin_memory=True).numpy()
    Jpin = torch.empty(chunk, dtype=torch.int64, pin_memory=True).numpy()
    Zpin = torch.empty((chunk, wl.device.Z), dtype=torch.int64, pin_memory=True).numpy()
    e2e_first = sim.t
    MG.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        first = sim.t
        Vpin[:] = wl.V[first:first + chunk]
        kmc_set_voltage(sim.h, first, Vpin)
        sim.step_n(chunk)
        kmc_observables(sim.h, first, chunk, Jpin, Zpin, None)
    torch.cuda.synchronize()
    e2e_s = MG.max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = MG.whole_job_rate(units, e2e_s)
    e2e_last = sim.t

    if rank == 0:
        hbm, hbm_src, sm_max = _peaks()
        draws = float(cnt1[0] - cnt0[0]) / args.steps        # Philox blocks per launch
        per_launch_s = (ms_rank / args.steps) / 1e3
        alu_peak = SMS * IMAD_PER_SM_PER_CLK * sm_max * 1e6 / PHILOX_IMAD_SLOTS / 1e9  # G blocks/s
        achieved = draws / per_launch_s / 1e9
        from paper_2511_09413_gb300.kmc import kmc_philox_probe
        probe = kmc_philox_probe(stream.cuda_stream) / 1e9
        hbm_achieved = BYTES_PER_SITE_UPDATE * su_per_step / per_launch_s / 1e9
        cyc = (t_last - t_first) / 100000.0
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name if world == 1 else "hysteresis_%dx%d" % (
                           args.rails * (world if args.scaling == "weak" else 1), L),
                       "rails": R * world if args.scaling == "weak" else args.rails,
                       "rails_per_gpu": R, "sites": L,
                       "time_steps_per_step": chunk, "site_updates_per_step": su_per_step * world
                       if args.scaling == "weak" else args.rails * L * chunk,
                       "timed_time_steps": [t_first, t_last],
                       "timed_protocol_cycles": cyc,
                       "e2e_time_steps": [e2e_first, e2e_last],
                       "fill": wl.fill,
                       "electrodes": "injecting/extracting 1e9 Hz", "barriers": "per site N(0.40, 0.02) eV",
                       "protocol": "triangle +-2 V, 1e5 steps/cycle",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": ("rails partitioned over %d GPUs (rail_base), %s scaling" % (
                           world, args.scaling)) if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "G Philox4x32-10 blocks/s", "frac": achieved / alu_peak,
                         "traffic": _traffic_per_launch(R, chunk),
                         "traffic_unit": "DRAM bytes per launch (ncu, scaled by rails)",
                         "peak_basis": "%d SMs x %d IMAD lanes/clk x %.0f MHz / %d IMAD issue slots "
                                       "per block" % (SMS, IMAD_PER_SM_PER_CLK, sm_max,
                                                      PHILOX_IMAD_SLOTS),
                         "philox_only_probe": {"achieved": probe, "frac_of_peak": probe / alu_peak,
                                               "sweep_frac_of_probe": achieved / probe,
                                               "basis": "kmc_philox_probe: the draw loop's Philox "
                                                        "blocks alone, measured in this run"},
                         "hbm_basis": {"achieved_GBps": hbm_achieved,
                                       "peak_GBps": hbm, "peak_source": hbm_src,
                                       "frac": hbm_achieved / hbm,
                                       "bytes_per_site_update": BYTES_PER_SITE_UPDATE}},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": args.steps,
                    "h2d_bytes_per_step": int(Vpin.nbytes),
                    "d2h_bytes_per_step": int(Jpin.nbytes + Zpin.nbytes)},
            # per timed step: one sweep_kernel launch and one zone_scan_kernel launch
            "gpu_launches": 2 * args.steps,
            "counters": {"philox_blocks_per_site_update": draws / su_per_step,
                         "fp64_decisions": int(cnt1[1] - cnt0[1]),
                         "moves": int(cnt1[2] - cnt0[2])},
            "wall_s": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget)
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched STDP devices (512 by default) in one persistent launch per chunk,
    against the same devices advanced one after another by the single-device
    kernel: equal work, hence equal ensemble error."""
    import torch
    from paper_2511_09413_gb300 import kmc

    torch.cuda.set_device(0)
    kmc.load()
    chunk = args.chunk
    n_steps = (args.warmup + args.steps) * chunk + args.probe
    devs, Vs, fills, delays = W.stdp_batch(args.instances, n_steps=n_steps)
    n = len(devs)
    sites = sum(d.R * d.L for d in devs)
    stream = torch.cuda.current_stream()
    b = kmc.Batch(devs, Vs, [1] * n, fills=fills, stream=stream.cuda_stream)
    warps, spl = b.tune(args.probe)
    acc = b.accept_path
    for _ in range(args.warmup):
        b.step_n(chunk)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.step_n(chunk)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    value = sites * chunk * args.steps / (ms / 1e3)
    b.close()
    # the same devices, one at a time, single-device kernel
    plain_ms = 0.0
    for d, V, f in zip(devs, Vs, fills):
        sim = kmc.Sim(d, V, init_mode=1, fill=f, stream=stream.cuda_stream)
        sim.step_n(chunk)                      # warm-up
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        sim.step_n(chunk)
        a1.record(stream)
        a1.synchronize()
        plain_ms += a0.elapsed_time(a1)
        sim.close()
    plain_value = sites * chunk / (plain_ms / 1e3)
    line = {
        "metric": METRIC + ", batched", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "stdp_batch", "devices": n, "sites_total": sites,
                   "rails": "log-uniform [256, 16384]", "sites_per_rail": "log-uniform [128, 2048]",
                   "fill": "U(0.05, 0.4)", "protocol": "spike pair, 1 V 1 ms pulses, 2000 steps/ms",
                   "time_steps_per_step": chunk, "tuned": {"warps_per_cta": warps,
                                                           "steps_per_launch": spl,
                                                           "accept_path": acc}},
        "plain_one_device_at_a_time": {"value": plain_value, "unit": UNIT,
                                       "speedup_batched": value / plain_value},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """Likelihood-ratio gradient of the mean relaxation current per replica
    with respect to (Ea, nu, kappa, fill): 256 replicas of 4,096 x 512, 1 V x
    1e4 steps then 5e4 relaxation steps.  Times the forward run and the
    backward pass (kmc_grad).  With --fd-groups G > 0 it also compares, on
    --fd-replicas replicas split into G independent groups, the LR gradient
    with central differences (h = 1e-3 relative) under common random numbers,
    and reports the GPU time each needs for equal standard error."""
    import torch
    from paper_2511_09413_gb300 import kmc

    torch.cuda.set_device(0)
    kmc.load()
    stream = torch.cuda.current_stream()
    n_write, n_relax = args.adj_write, args.adj_relax

    def weights(replicas):
        w = np.zeros(n_write + n_relax)
        w[n_write:] = 1.0 / (n_relax * replicas)
        return w

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    def run(replicas, instance, theta=None):
        wl = W.adjoint_relaxation(replicas=replicas, n_write=n_write, n_relax=n_relax,
                                  instance=instance)
        d = wl.device
        fill = wl.fill
        if theta is not None:
            d.Ea, d.nu, d.kappa, fill = theta
        return wl, d, fill

    # warm-up on a small device (loads the kernels, sets the allocator pools)
    wl, d, fill = run(1, 0)
    sim = kmc.Sim(d, wl.V, 1, fill=fill, stream=stream.cuda_stream)
    sim.step_n(200)
    sim.grad(weights(1)[:200], None)
    sim.close()

    wl, d, fill = run(args.replicas, 0)
    sim = kmc.Sim(d, wl.V, 1, fill=fill, stream=stream.cuda_stream)
    n = wl.n_steps
    _, t_fwd = timed(lambda: sim.step_n(n))
    (g, se), t_bwd = timed(lambda: sim.grad(weights(args.replicas), None))
    J, _ = sim.traces()
    sim.close()
    su = d.R * d.L * n
    names = ["Ea", "nu", "kappa", "fill"]
    line = {
        "metric": METRIC + ", adjoint", "value": su / (t_fwd + t_bwd), "unit": UNIT,
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * (t_fwd + t_bwd),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "replicas": args.replicas, "rails_per_replica": 4096,
                   "sites": d.L, "fill": wl.fill, "dt_s": d.dt, "write": "1 V x %d steps" % n_write,
                   "relaxation_steps": n_relax,
                   "observable": "mean relaxation current per replica (ions/step)",
                   "value_basis": "site-updates of the forward run / (forward + backward time)"},
        "forward": {"site_updates_per_s": su / t_fwd, "s": t_fwd},
        "backward": {"site_updates_per_s": su / t_bwd, "s": t_bwd},
        "observable": float(J[n_write:].mean() / args.replicas),
        "grad": dict(zip(names, g.tolist())), "grad_stderr": dict(zip(names, se.tolist())),
        # standard error relative to the estimate, and the replicas at which it
        # would reach 5 % (it falls as 1 / sqrt(replicas): replicas are independent)
        "grad_rel_stderr": dict(zip(names, (se / np.abs(g)).tolist())),
        "replicas_for_5pct_stderr": dict(zip(names, np.ceil(
            args.replicas * (se / np.abs(g) / 0.05) ** 2).astype(int).tolist())),
    }
    if args.fd_groups > 0:
        G = args.fd_groups
        per = max(1, args.fd_replicas // G)
        lr, fd, t_lr, t_f = [], [], 0.0, 0.0
        for grp in range(G):
            wl, d, fill = run(per, 1000 + grp)
            theta = [d.Ea, d.nu, d.kappa, fill]
            sim = kmc.Sim(d, wl.V, 1, fill=fill, stream=stream.cuda_stream)
            _, t1 = timed(lambda: sim.step_n(n))
            (gg, _), t2 = timed(lambda: sim.grad(weights(per), None))
            sim.close()
            lr.append(gg)
            t_lr += t1 + t2
            row = []
            for k in range(4):
                h = 1e-3 * abs(theta[k])
                vals = []
                for sgn in (1.0, -1.0):
                    th = list(theta)
                    th[k] += sgn * h
                    wl2, d2, fill2 = run(per, 1000 + grp, th)
                    s2 = kmc.Sim(d2, wl2.V, 1, fill=fill2, stream=stream.cuda_stream)
                    _, t3 = timed(lambda: s2.step_n(n))
                    t_f += t3
                    J2, _ = s2.traces()
                    s2.close()
                    vals.append(J2[n_write:].mean() / per)
                row.append((vals[0] - vals[1]) / (2 * h))
            fd.append(row)
        lr, fd = np.array(lr), np.array(fd)
        lm, ls = lr.mean(0), lr.std(0, ddof=1) / np.sqrt(G)
        fm, fs = fd.mean(0), fd.std(0, ddof=1) / np.sqrt(G)
        cost_lr = t_lr / G                  # one forward + one backward: all four entries
        cost_fd = t_f / G / 4               # two forwards: one entry
        line["fd_check"] = {
            "replicas": per * G, "groups": G, "h_relative": 1e-3,
            "lr": dict(zip(names, lm.tolist())), "lr_stderr": dict(zip(names, ls.tolist())),
            "fd": dict(zip(names, fm.tolist())), "fd_stderr": dict(zip(names, fs.tolist())),
            "z": dict(zip(names, ((lm - fm) / np.hypot(ls, fs)).tolist())),
            "rel_diff": dict(zip(names, (np.abs(lm - fm) / np.abs(fm)).tolist())),
            # the full-size LR estimate against the differences of the check
            "lr_full_rel_diff": dict(zip(names, (np.abs(g - fm) / np.abs(fm)).tolist())),
            "lr_full_z": dict(zip(names, ((g - fm) / np.hypot(se, fs)).tolist())),
            "gpu_s_per_group": {"lr_forward_backward": cost_lr, "fd_two_forwards": cost_fd},
            # GPU time for one entry at equal standard error: FD / LR
            "fd_over_lr_time_at_equal_error": dict(zip(names, (
                (cost_fd * fs ** 2) / (cost_lr * ls ** 2)).tolist())),
        }
    print(json.dumps(line), flush=True)
    return 0


def run_stdp(args):
    """STDP curve of the batched devices: the 512 spike-pair devices over their
    whole 120 ms window in one batched run (rail counts divided by
    --stdp-rail-div to bound the time; the rails are independent, so this
    changes only the ensemble size), and per device the conductance change
    dG = G(end) - G(just before the pre pulse), G = decile-1 ions / ions."""
    import torch
    from paper_2511_09413_gb300 import kmc

    torch.cuda.set_device(0)
    kmc.load()
    devs, Vs, fills, delays = W.stdp_batch(args.instances)
    div = max(1, args.stdp_rail_div)
    devs = [dataclasses.replace(d, R=max(16, d.R // div)) for d in devs]
    n = len(Vs[0])
    t_pre = int(round(55.0 * 2000))
    stream = torch.cuda.current_stream()
    b = kmc.Batch(devs, Vs, [1] * len(devs), fills=fills, stream=stream.cuda_stream)
    b.set_launch(8, 1024)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step_n(n - 1)
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    dG = np.zeros(len(devs))
    for i in range(len(devs)):
        _, Zp = b.traces(i, t_pre, 1)           # zone counts at the start of the pre pulse
        _, Ze = b.traces(i, n - 2, 1)           # ... and at the start of the last step
        N = float(Zp[0].sum())
        dG[i] = (Ze[0, 0] - Zp[0, 0]) / max(N, 1.0)
    b.close()
    delays = np.asarray(delays)
    edges = np.linspace(-50, 50, 11)
    curve = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (delays >= lo) & (delays < hi)
        curve.append({"dt_ms": [float(lo), float(hi)], "devices": int(m.sum()),
                      "dG_mean": float(dG[m].mean()) if m.any() else None,
                      "dG_sem": float(dG[m].std(ddof=1) / np.sqrt(m.sum())) if m.sum() > 1 else None})
    sites = sum(d.R * d.L for d in devs)
    line = {
        "metric": METRIC + ", batched STDP curve", "value": sites * (n - 1) / secs, "unit": UNIT,
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * secs, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "stdp_batch", "devices": len(devs), "sites_total": sites,
                   "rail_divisor": div, "time_steps": n - 1,
                   "protocol": "spike pair, 1 V 1 ms pulses, t_pre = 55 ms, 2000 steps/ms",
                   "dG": "G(120 ms) - G(55 ms^-), G = decile-1 ions / ions"},
        "stdp_curve": curve,
        "per_device": {"dt_ms": delays.round(3).tolist(), "dG": dG.round(6).tolist()},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_fit(args):
    """Batched + adjoint fit: gradient descent on (Ea, kappa) for 256 devices
    of 2,048-8,192 rails x 256-1,024 sites under a potentiation/forgetting
    protocol, toward the oracle's curves at the hidden (0.42 eV, 0.9) stored
    in tests/golden.  Each iteration is one batched forward run and one
    backward pass per device."""
    import torch
    from paper_2511_09413_gb300 import kmc
    from paper_2511_09413_gb300.fit import MaterialFit

    torch.cuda.set_device(0)
    kmc.load()
    name = os.path.join(ROOT, "tests", "golden", "fit_target_%ddev_%dp_%df.npz" % (
        args.fit_devices, args.fit_pulses, args.fit_forget))
    tgt = np.load(name)
    devs, V, fills, samples = W.fit_batch(args.fit_devices, n_pulses=args.fit_pulses,
                                          forget_steps=args.fit_forget)
    assert np.array_equal(samples, tgt["sample_steps"])
    fit = MaterialFit(devs, V, fills, samples, tgt["target"],
                      stream=torch.cuda.current_stream().cuda_stream)
    if args.fit_eval or args.fit_loss:
        return _fit_evaluations(args, fit, devs, tgt, name)
    hist = fit.run(0.40, 1.0, iters=args.fit_iters, lr=(6e-3, 5e-2))
    su = sum(d.R * d.L for d in devs) * fit.n_steps
    t_f = sum(h.seconds_forward for h in hist)
    t_b = sum(h.seconds_backward for h in hist)
    last = hist[-1]
    Ea_h, k_h = float(tgt["Ea"]), float(tgt["kappa"])
    line = {
        "metric": METRIC + ", batched + adjoint fit", "value": su * len(hist) / (t_f + t_b),
        "unit": UNIT, "n_gpus": 1, "steps": len(hist), "warmup": 0,
        "ms_per_step": 1e3 * (t_f + t_b) / len(hist), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fit_batch", "devices": len(devs),
                   "sites_total": sum(d.R * d.L for d in devs),
                   "protocol": "%d pulses of 0.8 V x 0.5 ms, 0.5 ms apart, then %d steps" % (
                       args.fit_pulses, args.fit_forget),
                   "time_steps": fit.n_steps, "samples_per_curve": len(samples),
                   "target": os.path.relpath(name, ROOT) + " (oracle, %d rails per device)" % int(
                       tgt["rails_per_device"]),
                   "hidden": {"Ea": Ea_h, "kappa": k_h},
                   "value_basis": "forward site-updates per evaluation / (forward + backward time)"},
        "forward_site_updates_per_s": su * len(hist) / t_f,
        "backward_site_updates_per_s": su * len(hist) / t_b,
        "history": [{"Ea": h.Ea, "kappa": h.kappa, "loss": h.loss,
                     "grad": h.grad.tolist(), "grad_stderr": h.stderr.tolist(),
                     "s_forward": h.seconds_forward, "s_backward": h.seconds_backward}
                    for h in hist],
        "final": {"Ea": last.Ea, "kappa": last.kappa,
                  "Ea_rel_error": abs(last.Ea - Ea_h) / Ea_h,
                  "kappa_rel_error": abs(last.kappa - k_h) / k_h},
    }
    print(json.dumps(line), flush=True)
    return 0


def _points(spec):
    return [tuple(float(x) for x in p.split(",")) for p in spec.split(";") if p.strip()]


def _fit_evaluations(args, fit, devs, tgt, name):
    """Loss and gradient (--fit-eval) or loss alone (--fit-loss) of the fit
    at given (Ea, kappa) points, without iterating: whether the curves of the
    protocol determine the hidden parameters."""
    su = sum(d.R * d.L for d in devs) * fit.n_steps
    evals = []
    for Ea, ka in _points(args.fit_eval):
        st = fit.loss_and_grad(Ea, ka)
        evals.append({"Ea": Ea, "kappa": ka, "loss": st.loss, "grad": st.grad.tolist(),
                      "grad_stderr": st.stderr.tolist(), "s_forward": st.seconds_forward,
                      "s_backward": st.seconds_backward,
                      "forward_site_updates_per_s": su / st.seconds_forward,
                      "backward_site_updates_per_s": su / st.seconds_backward})
    losses = []
    for Ea, ka in _points(args.fit_loss):
        loss, G, sec = fit.loss(Ea, ka)
        losses.append({"Ea": Ea, "kappa": ka, "loss": loss, "s_forward": sec,
                       "forward_site_updates_per_s": su / sec,
                       "G_end_mean": float(G[:, -1].mean()),
                       "G_peak_mean": float(G.max(axis=1).mean())})
    secs = sum(e["s_forward"] + e.get("s_backward", 0.0) for e in evals + losses)
    line = {
        "metric": METRIC + ", batched + adjoint fit evaluations", "value": su * len(evals + losses) / secs,
        "unit": UNIT, "n_gpus": 1, "steps": len(evals + losses), "warmup": 0,
        "ms_per_step": 1e3 * secs / max(1, len(evals + losses)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fit_batch", "devices": len(devs),
                   "sites_total": sum(d.R * d.L for d in devs),
                   "protocol": "%d pulses of 0.8 V x 0.5 ms, 0.5 ms apart, then %d steps" % (
                       args.fit_pulses, args.fit_forget),
                   "time_steps": fit.n_steps, "samples_per_curve": len(fit.sample_steps),
                   "target": os.path.relpath(name, ROOT) + " (oracle, %d rails per device)" % int(
                       tgt["rails_per_device"]),
                   "hidden": {"Ea": float(tgt["Ea"]), "kappa": float(tgt["kappa"])}},
        "evaluations": evals, "losses": losses,
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["kmc", "reference"], default="kmc")
    ap.add_argument("--workload", choices=["hysteresis", "batched", "adjoint", "fit", "stdp"],
                    default="hysteresis")
    ap.add_argument("--stdp-rail-div", type=int, default=16, help="stdp: rails divided by this")
    ap.add_argument("--fit-devices", type=int, default=256)
    ap.add_argument("--fit-pulses", type=int, default=8)
    ap.add_argument("--fit-forget", type=int, default=8000)
    ap.add_argument("--fit-iters", type=int, default=5)
    ap.add_argument("--fit-eval", default="", help="fit: 'Ea,kappa;...' points for loss and gradient")
    ap.add_argument("--fit-loss", default="", help="fit: 'Ea,kappa;...' points for the loss alone")
    ap.add_argument("--replicas", type=int, default=256, help="replicas in the adjoint workload")
    ap.add_argument("--adj-write", type=int, default=10000, help="write-pulse steps (adjoint)")
    ap.add_argument("--adj-relax", type=int, default=50000, help="relaxation steps (adjoint)")
    ap.add_argument("--fd-groups", type=int, default=0, help="adjoint: groups of the FD check")
    ap.add_argument("--fd-replicas", type=int, default=32, help="adjoint: replicas of the FD check")
    ap.add_argument("--instances", type=int, default=512, help="devices in the batched workload")
    ap.add_argument("--probe", type=int, default=1024, help="autotuner probe steps (batched)")
    ap.add_argument("--chunk", type=int, default=10000, help="time steps per benchmark step")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="N > 1: each rank its own 65,536 rails (weak) or a share of them (strong)")
    ap.add_argument("--rails", type=int, default=65536)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-steps", type=int, default=10, help="oracle time steps per reference step")
    ap.add_argument("--ref-stride", type=int, default=16, help="oracle samples every n-th rail")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "kmc" and not os.environ.get("KMC_BENCH_ALLOW_FEW_WARMUP"):
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "fit":
        return run_fit(args)
    if args.workload == "stdp":
        return run_stdp(args)
    return run_kmc(args)


if __name__ == "__main__":
    sys.exit(main())
