#!/usr/bin/env python3
"""DPD fluid-step benchmark on GB300: particle-steps/s.

Workload (default): one periodic box L = 128 rc, rho = 3 (6,291,456
particles), a = 25, gamma = 4.5, kT = 1, dt = 0.005, seeded uniform positions
and Maxwellian velocities.  A step is the whole hot path: kick/drift/wrap and
cell count, scan, stable reorder, pair forces with the Philox pair noise.

  value     particle-steps/s with the state resident in HBM (CUDA events on the
            library's stream around K steps, max over ranks)
  e2e       the same metric through the C ABI with host buffers: upload from
            pinned memory, K steps each followed by a statistics read-back,
            download of the final state
  roofline  the force kernel against the FP32/INT32 issue peak
            (SMs x 128 lanes x SM clock), timed with per-stage events
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample
  batched, served, mixture, paper_benchmark
            the 512-box mix, the served request stream, a binary mixture,
            and the paper's own benchmark box (L = 64, rho = 8), each with
            its own workload description

`--impl reference` times the oracle alone (the reference arm of this build).
With --gpus N > 1 (torchrun) every rank steps its own independent replica.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DPD particle-steps/s on 1 GB300, batched vs one-box-at-a-time; p50/p99 latency"
UNIT = "particle-steps/s"

# Algorithmic ALU work of the force stage per particle-step, with each
# candidate and each interacting pair counted once (what Newton's third law
# leaves to do): 27 rho / 2 candidates and (4 pi / 3) rho / 2 pairs.  A
# candidate test is 7 FP32-pipe instructions (3 subtractions, a multiply and
# two fused multiply-adds for r^2, one compare); a pair is 30 FP32-pipe
# instructions (r, w, e . v_ij, the three terms, the update, the noise map)
# plus one Philox-4x32-10 word.  The roofline weighs the Philox word by the
# measured issue rates: FMA-equivalent work = FP32 instructions + words x
# (FMA rate / Philox word rate), against the measured FMA rate.  (An
# unweighted count for comparison: 7 slots per candidate and 110 per pair --
# 30 FP32 and 80 integer -- against SMs x 128 lanes x clock.)
CAND_SLOTS = 7
PAIR_FP32 = 30
UNWEIGHTED_PAIR_SLOTS = 110


def force_counts(rho: float):
    cands = 27.0 * rho / 2.0                 # 27-cell stencil, each pair once
    pairs = (4.0 * math.pi / 3.0) * rho / 2.0
    return cands, pairs


def force_slots_per_particle(rho: float) -> float:
    """The unweighted count (lane-instruction slots per particle)."""
    cands, pairs = force_counts(rho)
    return cands * CAND_SLOTS + pairs * UNWEIGHTED_PAIR_SLOTS


def force_fma_equiv_per_particle(rho: float, fma_rate: float, philox_rate: float) -> float:
    """FMA-equivalent work per particle with the Philox word weighed by the
    measured rates."""
    cands, pairs = force_counts(rho)
    return cands * CAND_SLOTS + pairs * (PAIR_FP32 + fma_rate / philox_rate)


# FP32 flops (an FMA counts 2) of the same work: a candidate's distance test
# (3 subtractions, a multiply and two FMAs) and an interacting pair's r, w,
# e . v_ij, the three terms and the update, the noise map included.
CAND_FLOPS = 8
PAIR_FLOPS = 30


def force_flops_per_particle(rho: float) -> float:
    cands = 27.0 * rho / 2.0
    pairs = (4.0 * math.pi / 3.0) * rho / 2.0
    return cands * CAND_FLOPS + pairs * PAIR_FLOPS


# Algorithmic HBM bytes per particle-step of the streaming stages.  The
# full stencil orders each cell by previous slot (key pass + ranked
# reorder); the half stencil has no key pass and its reorder places by
# arrival rank and also zeroes the force it accumulates into.
STAGE_BYTES = {
    "full": {"integrate_bin": 48 + 32 + 8,   # read x, v, f; write x', v', cell, arrival rank
             "bin_keys": 8 + 4,              # read cell, rank; write key
             "bin_scatter": 8 + 32 + 32},    # read cell, start, x', v'; write x, v
    "half": {"integrate_bin": 48 + 32 + 8,
             "bin_scatter": 12 + 32 + 48},   # read cell, rank, start, x', v'; write x, v, f = 0
}


# DRAM traffic of the force kernel per launch and its L1 data-pipe
# throughput from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum; l1tex__data_pipe_lsu_wavefronts as a fraction of
# peak; profiles/force_direct_L128_rho3.md), valid only while the kernel
# sources and the tuning table (which picks the variant) hash to the value
# recorded with them.
TRAFFIC = {("half", 128.0, 3.0): (399.856e6, 0.780, "801e484dec6533db")}
KERNEL_SOURCES = ("paper_1911_04712_gb300/csrc/force.cu", "paper_1911_04712_gb300/csrc/force_direct.cuh",
                  "paper_1911_04712_gb300/csrc/dpd_device.cuh",
                  "paper_1911_04712_gb300/csrc/kernels.h", "paper_1911_04712_gb300/tuning_gb300.json")


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(L: float, rho: float, steps: int, seed: int = 0, threads: int = 0) -> dict:
    """The FP64 oracle (cell-list mode, OpenMP over the host cores, or
    `threads` of them) on a bounded sample: a box of the same recipe, `steps`
    steps after the initial force."""
    import oracle as O
    from paper_1911_04712_gb300.workloads import uniform_box_state
    x, v = uniform_box_state(L, rho=rho, seed=seed)
    p = O.Params(L=(L, L, L), a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=seed)
    prev = O.num_threads()
    if threads:
        O.set_num_threads(threads)
    try:
        cores = O.num_threads()
        st = O.State(p, x, v, mode=O.MODE_CELLS)
        t0 = time.perf_counter()
        st.run(steps)
        dt = time.perf_counter() - t0
    finally:
        O.set_num_threads(prev)
    return {"value": x.shape[0] * steps / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"L={L:g} box of the same recipe ({x.shape[0]} particles, rho={rho:g}), "
                      f"{steps} step(s) after the initial force, FP64 cell-list mode"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    L_sample = args.ref_L
    base = cpu_baseline(L_sample, args.rho, 1)   # warm the library and page in
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        cpu_baseline(L_sample, args.rho, 1, seed=1)
    t_steps = time.perf_counter()
    for k in range(args.steps):
        vals.append(cpu_baseline(L_sample, args.rho, 1, seed=2 + k)["value"])
    elapsed = time.perf_counter() - t_steps
    value = statistics.mean(vals)
    n = base["sample"]
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"oracle_sample_L{L_sample:g}_rho{args.rho:g}",
                   "sample_of": f"dpd_periodic_box_L{args.L:g}_rho{args.rho:g}",
                   "reference_sample_L": L_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                         "sample": n},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(out), flush=True)
    return 0


def run_batched(args, stream, world, rank):
    """512-box mix: one packed batch vs the same boxes one at a time with
    their own single-box contexts (same stream), both with states resident."""
    import torch

    import paper_1911_04712_gb300.batch as B
    import paper_1911_04712_gb300.dpd as dpd
    from paper_1911_04712_gb300.workloads import box_mix, uniform_box_state

    from paper_1911_04712_gb300.shard import shard_boxes
    specs = box_mix(args.nbox, master_seed=args.seed)
    if world > 1:                       # shard boxes over ranks, no data-path collective
        mine = shard_boxes([s.n * args.batch_steps for s in specs], rank, world)
        specs = [specs[k] for k in mine]
    states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=s.seed) for s in specs]
    n_tot = sum(len(x) for x, _ in states)
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    stencil = 1 if args.stencil == "half" else 0
    bt = B.Batch(descs, stream=stream, stencil=stencil)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    bt.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bt.step(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    stage_ms = bt.profile(10)
    bt.close()

    boxes = []
    for s, (x, v) in zip(specs, states):
        b = dpd.Box(s.L, a=s.a, gamma=s.gamma, kT=s.kT, rc=1.0, dt=s.dt, seed=s.seed, stream=stream,
                    stencil=stencil)
        b.set_state(x, v)
        b.step(args.warmup)
        boxes.append(b)
    torch.cuda.synchronize()
    e0.record(stream)
    for b in boxes:                      # one box at a time, each to completion
        b.step(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    for b in boxes:
        b.close()
    import torch.distributed as tdist
    from paper_1911_04712_gb300.shard import combine
    units, sec_b = combine(float(n_tot * args.batch_steps), ms_b / 1000.0, tdist, "cuda")
    _, sec_s = combine(float(n_tot * args.batch_steps), ms_s / 1000.0, tdist, "cuda")
    n_all, _ = combine(float(n_tot), 0.0, tdist, "cuda")
    rate_b = units / sec_b
    rate_s = units / sec_s
    n_tot = int(n_all)
    return {"workload": f"box mix: {args.nbox} boxes, L~U{{6..24}}, rho in {{3,4,5}}, "
                        f"a~U[10,80], gamma~U[2,8], kT~U[0.5,2], dt=0.005",
            "boxes": args.nbox, "particles": n_tot, "steps": args.batch_steps,
            "stencil": args.stencil,
            "value": rate_b, "unit": UNIT, "ms_per_step": ms_b / args.batch_steps,
            "one_box_at_a_time": {"value": rate_s, "ms_per_step": ms_s / args.batch_steps},
            "speedup_vs_one_at_a_time": rate_b / rate_s,
            "stages_ms": {k: round(t, 5) for k, t in zip(dpd.STAGE_NAMES, stage_ms)}}


def run_mixture(args, stream):
    """Binary mixture (species with their own a, gamma and cut-off per pair) on
    an L = 64 box against one species on the same box, same stencil."""
    import numpy as np
    import torch

    import paper_1911_04712_gb300.dpd as dpd
    from paper_1911_04712_gb300.workloads import uniform_box_state
    L, steps = args.mix_L, args.mix_steps
    x, v = uniform_box_state(L, rho=3.0, seed=args.seed + 7)
    n = len(x)
    species = (np.arange(n) % 2).astype(np.int32)
    a = np.array([[25.0, 40.0], [40.0, 25.0]])
    g = np.array([[4.5, 4.5], [4.5, 4.5]])
    rc = np.array([[1.0, 0.9], [0.9, 1.0]])
    stencil = 1 if args.stencil == "half" else 0
    out = {}
    for name in ("mixture", "one_species"):
        box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=args.seed,
                      stream=stream, stencil=stencil)
        if name == "mixture":
            box.set_species(a, g, rc)
            box.set_state(x, v, species=species)
        else:
            box.set_state(x, v)
        box.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        box.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": n * steps / (e0.elapsed_time(e1) / 1000.0), "ms_per_step": ms}
        box.close()
    return {"workload": f"binary mixture L={L:g} rho=3, 50/50, a = [[25, 40], [40, 25]], "
                        "gamma 4.5, rc = [[1, 0.9], [0.9, 1]]",
            "particles": n, "steps": steps, "stencil": args.stencil, "unit": UNIT,
            "value": out["mixture"]["value"], "ms_per_step": out["mixture"]["ms_per_step"],
            "one_species": out["one_species"],
            "kernel": "general force kernel (per-pair species tables)"}


def run_paper_benchmark(args, stream):
    """The paper's own benchmark (Sec. 5.1): one periodic box of L = 64 at
    rho = 8 (2,097,152 particles) driven by the periodic Poiseuille force,
    with the parameters of its weak-scaling runs (a = 50, gamma = 20, kT = 1,
    dt = 0.002).  Its figure on one P100 (7.01 ms per step, 2.99e8
    particle-steps/s) is context from other hardware, not a target."""
    import torch

    import paper_1911_04712_gb300.dpd as dpd
    from paper_1911_04712_gb300.workloads import uniform_box_state
    L, rho, steps = 64.0, 8.0, args.paper_steps
    x, v = uniform_box_state(L, rho=rho, seed=args.seed + 11)
    n = len(x)
    box = dpd.Box(L, a=50.0, gamma=20.0, kT=1.0, rc=1.0, dt=0.002, seed=args.seed,
                  stream=stream, stencil=1 if args.stencil == "half" else 0)
    box.set_param(dpd.PARAM_POISEUILLE_F, 0.05)
    box.set_state(x, v)
    box.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    box.close()
    return {"workload": "the paper's periodic-Poiseuille benchmark: L=64, rho=8, a=50, "
                        "gamma=20, kT=1, dt=0.002, periodic Poiseuille force f=0.05",
            "particles": n, "steps": steps, "stencil": args.stencil, "unit": UNIT,
            "value": n * steps / (ms * steps / 1000.0), "ms_per_step": ms,
            "paper": {"value": 2.99e8, "ms_per_step": 7.01, "hardware": "1x P100",
                      "note": "other hardware, context only"}}


def run_served(args, rank=0, world=1):
    """Prefix of the served request stream: Poisson arrivals submitted in real
    time to one continuous-batching queue per GPU under a 120 GB HBM budget
    (with N GPUs, requests go round-robin to the ranks' queues)."""
    import torch.distributed as tdist

    import paper_1911_04712_gb300.serve as S
    from paper_1911_04712_gb300.shard import gather_list, shard_requests
    from paper_1911_04712_gb300.workloads import request_stream

    reqs = request_stream(args.requests, rate=args.rate, master_seed=args.seed)
    reqs = [reqs[k] for k in shard_requests(len(reqs), rank, world)]
    q = S.Queue(int(120e9), chunk_steps=100, sample_every=20, nbins=16, policy=S.POLICY_FIFO,
                stencil=1 if args.stencil == "half" else 0)
    tickets = []
    t0 = time.perf_counter()
    for r in reqs:
        delay = t0 + r.t_arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(q.submit(S.make_request(r.L, rho=r.rho, a=r.a, gamma=r.gamma, kT=r.kT,
                                               dt=r.dt, seed=r.seed, steps=r.steps)))
    q.wait_all(3600)
    wall = time.perf_counter() - t0
    res = [q.result(t) for t in tickets]
    st = q.stats()
    q.close()
    lat = sorted(gather_list([x["latency"] for x in res], tdist))
    work = sum(gather_list([x["n"] * x["steps"] for x in res], tdist))
    span = max(gather_list([max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)],
                           tdist))
    kt_err = gather_list([abs(x["kT_mean"] / r.kT - 1) for x, r in zip(res, reqs)], tdist)
    failed = sum(gather_list([sum(1 for x in res if x["status"] != 0)], tdist))

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100 * (len(lat) - 1))))]

    # the same kind of runs one at a time with the plain single-box kernels:
    # the first `served_alone` requests of this rank, each to completion in
    # its own context on one stream (states of the same recipe)
    import torch
    import paper_1911_04712_gb300.dpd as dpd
    from paper_1911_04712_gb300.workloads import uniform_box_state
    stream = torch.cuda.current_stream()
    alone_work, alone_s = 0.0, 0.0
    for r in reqs[:args.served_alone]:
        x, v = uniform_box_state(r.L, rho=r.rho, kT=r.kT, seed=r.seed)
        b = dpd.Box(r.L, a=r.a, gamma=r.gamma, kT=r.kT, rc=1.0, dt=r.dt, seed=r.seed,
                    stream=stream, stencil=1 if args.stencil == "half" else 0)
        b.set_state(x, v)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(r.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        alone_s += e0.elapsed_time(e1) / 1000.0
        alone_work += float(len(x)) * r.steps
        b.close()
    alone_rate = alone_work / alone_s if alone_s > 0 else None

    return {"workload": f"first {args.requests} requests of the stream: Poisson {args.rate:g}/s, "
                        "L~lognormal(median 16, sigma 0.5) in [8,48], rho in {3,5}, "
                        "a~U[10,80], gamma~U[2,8], kT~U[0.5,2], steps~U{1000..20000}",
            "requests": len(lat), "failed": failed,
            "value": work / span, "unit": UNIT, "particle_steps": work,
            "p50_latency_s": pct(50), "p99_latency_s": pct(99), "max_latency_s": lat[-1],
            "wall_s": wall, "gpu_busy_s": st["busy_seconds"],
            "policy": "first come first served, admission at 100-step chunk boundaries",
            "stencil": args.stencil,
            "kT_mean_rel_err_median": statistics.median(kt_err),
            "one_request_at_a_time": {
                "value": alone_rate, "requests": min(args.served_alone, len(reqs)),
                "what": "the first requests' boxes, each run alone to its step count with the "
                        "plain single-box kernels (no sampling)"},
            "speedup_vs_one_at_a_time": (work / span / alone_rate) if alone_rate else None}


def run_native(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1911_04712_gb300 import build as _build
    if rank == 0 or world == 1:
        _build.build(philox_rounds=args.philox_rounds)
    if dist:
        dist.barrier()
    if args.philox_rounds != _build.PHILOX_ROUNDS:   # round-count study: that build instead
        os.environ["DPD_LIBRARY"] = _build.lib_path(args.philox_rounds)
    import paper_1911_04712_gb300.dpd as dpd
    from paper_1911_04712_gb300.workloads import uniform_box_state

    L, rho = args.L, args.rho
    x, v = uniform_box_state(L, rho=rho, seed=args.seed + rank)
    n = x.shape[0]
    stream = torch.cuda.current_stream()
    tiling = dict(tiles=args.tiles, tile_cells=args.tile_cells, stage_cap=args.stage_cap)
    if args.variant is not None:
        tiling["variant"] = args.variant
    box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=args.seed + rank,
                  stencil=(1 if args.stencil == "half" else 0), stream=stream, **tiling)
    box.set_state(x, v)
    box.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()

    clocks = ClockSampler(local).start() if not args.no_clocks else None
    # measured issue rates for the force kernel's roofline, then about a
    # second of untimed steps so that the clock samples see the GPU under
    # this load through the timed region
    rates = dpd.issue_rates(stream)
    if clocks:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 1.0:
            box.step(20)
            torch.cuda.synchronize()
    # ---- device-resident timed region
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # ---- per-stage events (same workload, same stream) for the roofline
    stage_ms = box.profile(args.steps)
    clk = clocks.stop() if clocks else None
    if clk:
        clk["window"] = "sampled every 200 ms from before a 1 s untimed load through the timed region and the per-stage profile"
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * args.steps * world / (ms / 1000.0)

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median")
    clock_src = "median SM clock sampled under load"
    if not (clk or {}).get("sm_mhz"):
        clock_src = "median SM clock under load from MEASURED_PEAKS.json"
    lane_peak = sms * 128 * float(sm_mhz) * 1e6 / 1e12 if sm_mhz else None   # T lane-ops/s
    force_ms = stage_ms[4]
    force_s = force_ms / 1000.0
    traffic = None
    l1_frac = None
    rec = TRAFFIC.get((args.stencil, float(L), float(rho)))
    if rec and rec[2] == kernel_hash() and args.philox_rounds == 10:
        traffic, l1_frac = rec[0], rec[1]
    fma_rate, phx_rate = rates["fma_lane_ops_per_s"], rates["philox_words_per_s"]
    work = force_fma_equiv_per_particle(rho, fma_rate, phx_rate) * n
    achieved = work / force_s / 1e12
    peak = fma_rate / 1e12
    unweighted_achieved = force_slots_per_particle(rho) * n / force_s / 1e12
    fp32_achieved = force_flops_per_particle(rho) * n / force_s / 1e12
    fp32_peak = 2.0 * peak
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    stages = {}
    for name, t in zip(dpd.STAGE_NAMES, stage_ms):
        d = {"ms": round(t, 5), "share": round(t / sum(stage_ms), 4)}
        if name in STAGE_BYTES[args.stencil]:
            gbs = STAGE_BYTES[args.stencil][name] * n / (t / 1000.0) / 1e9
            d.update({"GB/s": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 3)})
        stages[name] = d

    # ---- the other stencil on the same state, for the half-vs-full comparison
    other = "full" if args.stencil == "half" else "half"
    obox = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=args.seed + rank,
                   stencil=(1 if other == "half" else 0), stream=stream)
    obox.set_state(x, v)
    obox.step(args.warmup)
    ostage = obox.profile(min(args.steps, 50))
    obox.close()
    stencils = {args.stencil: {"force_ms": round(stage_ms[4], 5), "step_ms": round(sum(stage_ms), 5),
                               "deterministic": args.stencil == "full"},
                other: {"force_ms": round(ostage[4], 5), "step_ms": round(sum(ostage), 5),
                        "deterministic": other == "full"}}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hp = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        hv = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        hp.numpy()[:] = x
        hv.numpy()[:] = v
        ebox = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=args.seed + rank,
                       stencil=(1 if args.stencil == "half" else 0), stream=stream, **tiling)
        ebox.set_state(hp.numpy(), hv.numpy())      # warm allocation
        ebox.step(2)
        ebox.stats()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ebox.set_state(hp.numpy(), hv.numpy())
        for _ in range(args.steps):
            ebox.step(1)
            ebox.stats()
        ebox.get_state_into(hp.numpy(), hv.numpy())
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": n * args.steps * world / el, "unit": UNIT,
               "h2d_bytes_per_step": int(round(24 * n / args.steps)),
               "d2h_bytes_per_step": int(round(24 * n / args.steps)) + 64,
               "what": "set_state from pinned host, K x (step + FP64 stats read-back), "
                       "get_state to pinned host"}
        ebox.close()

    batched = None
    if not args.no_batched:
        batched = run_batched(args, stream, world, rank)

    served = None
    if not args.no_served:
        served = run_served(args, rank, world)

    mixture = None
    if not args.no_mixture:
        mixture = run_mixture(args, stream)

    paper = None
    if not args.no_paper_benchmark:
        paper = run_paper_benchmark(args, stream)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.cpu_L, rho, args.cpu_steps)
        base["single_core"] = cpu_baseline(32.0, rho, 3, threads=1)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"dpd_periodic_box_L{L:g}_rho{rho:g}", "particles": n,
                       "L": L, "rho": rho, "a": 25.0, "gamma": 4.5, "kT": 1.0, "dt": 0.005,
                       "stencil": args.stencil, "force_tiles": box.tiling(),
                       "philox_rounds": dpd.philox_rounds(),
                       "l2": "state larger than L2 "
                       f"({48 * n / 1e6:.0f} MB of float4 x, v, f)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "alu", "kernel": "force", "achieved": achieved,
                         "peak": peak, "unit": "T FMA-equivalent lane-ops/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "l1_pipe_frac": l1_frac,
                         "peak_from": "measured on this GPU by dpd_issue_rates: FP32 FMA "
                                      f"{fma_rate / 1e12:.2f} T lane-ops/s, Philox-4x32-10 "
                                      f"{phx_rate / 1e12:.4f} T words/s (1 word = "
                                      f"{fma_rate / phx_rate:.1f} FMA slots)",
                         "work_per_particle": force_fma_equiv_per_particle(rho, fma_rate, phx_rate),
                         "unweighted_count": {"achieved": unweighted_achieved, "peak": lane_peak,
                                          "unit": "T lane-ops/s",
                                          "frac": (unweighted_achieved / lane_peak) if lane_peak else None,
                                          "peak_from": f"{sms} SMs x 128 lanes x {sm_mhz} MHz "
                                                       f"({clock_src})"},
                         "fp32": {"achieved": fp32_achieved, "peak": fp32_peak,
                                  "unit": "TFLOP/s", "frac": fp32_achieved / fp32_peak}},
            "stages": stages,
            "stencils": stencils,
            "gpu_launches": dpd.kernels_per_step(args.stencil == "half") * args.steps,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": base,
            "batched": batched,
            "served": served,
            "mixture": mixture,
            "paper_benchmark": paper,
        }
        print(json.dumps(out), flush=True)
    box.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--L", type=float, default=128.0)
    ap.add_argument("--rho", type=float, default=3.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--stencil", choices=("full", "half"), default="half")
    ap.add_argument("--tiles", type=int, default=None, help="1: staged force tiles, 0: direct")
    ap.add_argument("--tile-cells", type=int, default=None)
    ap.add_argument("--variant", type=int, default=None, help="force-kernel variant (default: tuned)")
    ap.add_argument("--stage-cap", type=int, default=None)
    ap.add_argument("--cpu-L", type=float, default=64.0)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--ref-L", type=float, default=32.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-mixture", action="store_true")
    ap.add_argument("--no-paper-benchmark", action="store_true")
    ap.add_argument("--paper-steps", type=int, default=200)
    ap.add_argument("--mix-L", type=float, default=64.0)
    ap.add_argument("--mix-steps", type=int, default=200)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--served-alone", type=int, default=16,
                    help="requests of the served stream also run one at a time")
    ap.add_argument("--nbox", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--philox-rounds", type=int, default=10,
                    help="noise generator rounds (10; others only for a round-count study)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
