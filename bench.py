#!/usr/bin/env python3
"""Benchmark of the exact passing-point search on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pps|reference]

One step = one pass of the whole search (state staging, intercept times,
ball times, margins, shot angles, scores, mask, argmax) over one batch of
the batched workload: 4096 seeded SSL-shaped states, 12 x 9 m field, 0.05 m
grid (241 x 181 receive points), kick speeds {2, 3.5, 5, 6.5} m/s, K = 64
samples per pass, 8 opponents.  Metric: pass-candidate evaluations per
second, states x points x speeds x opponents / time.

Under torchrun each rank searches its own 4096 states (weak scaling, no
data-path collective); the barrier and the max over ranks of the timed
region are the only cross-rank traffic.  Rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on the host cores instead,
each step a bounded sample (16 states) of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pass-candidate evals/s (state×pt×speed×opp)"
UNIT = "evals/s"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
CPU_SAMPLE_STATES = 32       # oracle sample for the cpu_baseline key
REF_SAMPLE_STATES = 16       # oracle sample per step of --impl reference

# Algorithmic work of the formulation the kernel evaluates (FP32 lane-ops,
# an FMA counted once; MUFU ops counted separately):
#   per opponent interaction (state, point, sample, opponent): 14 FP32 + 2 MUFU
#   per ball evaluation (state, point, sample, speed):          3 FP32 + 1 MUFU
OPS_INTERACTION, MUFU_INTERACTION = 14, 2
OPS_BALL, MUFU_BALL = 3, 1
# The plan's per-unit estimate made before the kernel existed: about 20 FP32
# lane-ops per interaction and 8 per ball evaluation (reported beside).
SURVEY_OPS_INTERACTION, SURVEY_OPS_BALL = 20, 8
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 32   # ncu: XU pipe peak ~1 warp-instr/clk/SM on GB300


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed, so
    that a comment edit does not count as a change of the kernel."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _kernel_src_digest():
    """Digest of the code (comments aside) the timed search kernel is built
    from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1909_07717_gb300", "csrc")
    for path in (os.path.join(csrc, "pps_search.cuh"),
                 os.path.join(csrc, "pps_lib.cu"),
                 os.path.join(ROOT, "include", "pps.h")):
        with open(path) as f:
            h.update((os.path.basename(path) + _code_only(f.read())).encode())
    return h.hexdigest()[:16]


def _profiled_traffic(digest):
    """DRAM bytes per launch of the search kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "search_kernel_batched.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_digest") == digest:
            return float(kv["dram_bytes_per_launch_full"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def _profile_kv(name):
    """The machine-readable "key: value" lines of a committed ncu summary."""
    kv = {}
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
    except OSError:
        pass
    return kv


def _alu_peak(nsm):
    """FP32 lane-ops/s: SMs x 128 FP32 lanes x the maximum SM clock."""
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    return nsm * FP32_LANES_PER_SM * sm_max * 1e6, sm_max


def _alu_roofline(ops, seconds, nsm, per_unit, units):
    peak, sm_max = _alu_peak(nsm)
    return {"bound": "alu", "achieved": ops / seconds / 1e12,
            "peak": peak / 1e12, "unit": "Tops/s (FP32 lane-ops)",
            "frac": ops / seconds / peak, "traffic": None,
            "ops_per_launch": ops, "per_unit": per_unit, "units": units,
            "peak_basis": (f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                           f"{sm_max:.0f} MHz (max SM clock)")}


def _oracle_pool_rate(jobs, threads):
    """Run oracle searches (callables) on `threads` host threads at once
    (each single-threaded; the calls release the interpreter); seconds."""
    import concurrent.futures as cf
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda f: f(), jobs))
    return time.perf_counter() - t0


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)
        return False

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _cpu_oracle_rate(w, batch, grid_spec, n_states, cores=None):
    """Oracle evals/s on the first n_states states, on `cores` threads (all
    host cores by default)."""
    import oracle
    from paper_1909_07717_gb300 import synth
    sub = synth.take(batch, list(range(n_states)))
    cores = cores or oracle.max_threads()
    t0 = time.perf_counter()
    oracle.search(sub, grid_spec, w.speeds, w.params, n_threads=cores)
    dt = time.perf_counter() - t0
    P = grid_spec[1] * grid_spec[2]
    evals = n_states * P * len(w.speeds) * w.n_opp
    return evals / dt, dt, cores


def _workload():
    from paper_1909_07717_gb300 import synth
    return synth.BATCHED


def _config(w, grid_nx, grid_ny, world, extra=None):
    cfg = {"workload": w.name, "states_per_gpu": w.n_states,
           "grid": [grid_nx, grid_ny], "spacing_m": w.spacing,
           "field_m": list(w.field), "speeds_mps": list(w.speeds),
           "K": w.K, "opponents": w.n_opp, "ball_decel": w.ball_decel,
           "vmax": w.vmax, "amax": w.amax, "seed": w.seed,
           "parallelism": f"state-sharded x{world} (replicas)",
           "l2": "flushed between timed steps (256 MiB write)"}
    cfg.update(extra or {})
    return cfg


def run_reference(args):
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    if rank != 0:
        return 0
    import oracle
    w = _workload()
    batch = w.states()
    nx, ny, x0, y0 = oracle.grid(w.field[0], w.field[1], np.float32(w.spacing))
    gs = (float(np.float32(w.spacing)), nx, ny, x0, y0)
    for _ in range(args.warmup):
        _cpu_oracle_rate(w, batch, gs, REF_SAMPLE_STATES)
    rates, times = [], []
    cores = 1
    for _ in range(args.steps):
        r, dt, cores = _cpu_oracle_rate(w, batch, gs, REF_SAMPLE_STATES)
        rates.append(r)
        times.append(dt)
    value = (REF_SAMPLE_STATES * nx * ny * len(w.speeds) * w.n_opp
             * len(times)) / sum(times)
    sample = (f"first {REF_SAMPLE_STATES} states of the batched workload "
              f"(seed {w.seed}) per step, full grid, all speeds")
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, nx, ny, 1, {"states_per_step":
                                            REF_SAMPLE_STATES}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_pps(args):
    import torch

    from paper_1909_07717_gb300 import build as pbuild
    from paper_1909_07717_gb300 import pps, shard, synth

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if world != args.gpus and world == 1 and args.gpus > 1:
        print("use torchrun for --gpus > 1", file=sys.stderr)
        return 2
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()

    if dist is not None:
        dist.barrier()
    w = _workload()
    if args.states:
        w.n_states = args.states
    # Rank r searches its own states (weak scaling, no shared data).
    seed = shard.rank_seed(w.seed, rank)
    batch = synth.ssl_states(seed, w.n_states, field_len=w.field[0],
                             field_wid=w.field[1], n_opp=w.n_opp, K=w.K,
                             ball_decel=w.ball_decel, vmax=w.vmax,
                             amax=w.amax)
    grid = pps.pps_grid_from_field(w.field[0], w.field[1], w.spacing)
    S, V, P, J = w.n_states, len(w.speeds), grid.nx * grid.ny, w.n_opp
    stream = torch.cuda.current_stream(dev)
    searcher = pps.Searcher(max_states=S, max_opp=J, device=local,
                            stream=stream)
    states_dev = searcher.states_to_device(batch)
    out = searcher.alloc_outputs(S, grid, V, mask=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    prm = pps.params_from_dict(w.params)

    def step():
        searcher.search(states_dev, S, grid, w.speeds, prm, out=out)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = shard.max_over_ranks(sum(step_ms), dist, dev)
    evals_per_step = S * P * V * J
    value = shard.job_rate(evals_per_step, world, args.steps, total_ms)

    # correctness guard on the measured output (cheap, after timing)
    best = pps.unpack_best(out["best"].cpu().numpy())
    if not np.all(best["status"] == 0):
        print("search reported inconsistent states", file=sys.stderr)
        return 3

    # ---- end to end through the C ABI with host (pinned) buffers
    rec = pps.pack_states(batch)
    h_states = torch.from_numpy(rec.view(np.uint8).copy()).pin_memory()
    h_best = torch.empty(S * 32, dtype=torch.uint8).pin_memory()
    words = pps.pps_mask_words(grid, V)
    h_mask = torch.empty(S * words, dtype=torch.int32).pin_memory()
    sp = np.asarray(w.speeds, np.float32)

    def step_host():
        pps.pps_search(searcher.ctx, h_states.data_ptr(), S, grid,
                       sp.ctypes.data, V, prm, h_best.data_ptr(),
                       h_mask.data_ptr(), None, 0)

    for _ in range(2):
        step_host()
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev2[i][0].record(stream)
        step_host()
        ev2[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2),
                                  dist, dev)
    e2e_value = shard.job_rate(evals_per_step, world, args.steps, e2e_ms)
    host_best = pps.unpack_best(h_best.numpy())
    if host_best.tobytes() != best.tobytes():
        print("host-buffer path disagrees with device path", file=sys.stderr)
        return 3

    line = None
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks = _peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        nsm = props.multi_processor_count
        interactions = S * P * w.K * J
        ball_evals = S * P * w.K * V
        ops = OPS_INTERACTION * interactions + OPS_BALL * ball_evals
        mufu = MUFU_INTERACTION * interactions + MUFU_BALL * ball_evals
        t_launch = (total_ms / args.steps) / 1e3
        peak_ops = nsm * FP32_LANES_PER_SM * sm_max * 1e6
        peak_mufu = nsm * MUFU_LANES_PER_SM * sm_max * 1e6
        digest = _kernel_src_digest()
        ops_survey = (SURVEY_OPS_INTERACTION * interactions
                      + SURVEY_OPS_BALL * ball_evals)
        prof = _profile_kv("search_kernel_batched.txt")
        ncu = None
        if "fma_pipe_active" in prof:
            ncu = {"fma_pipe_active": float(prof["fma_pipe_active"]),
                   "xu_pipe_active": float(prof["xu_pipe_active"]),
                   "source": "profiles/search_kernel_batched.txt",
                   "current_kernel": prof.get("kernel_source_digest") == digest}
        roof = {"bound": "alu", "achieved": ops / t_launch / 1e12,
                "peak": peak_ops / 1e12, "unit": "Tops/s (FP32 lane-ops)",
                "frac": ops / t_launch / peak_ops,
                "traffic": _profiled_traffic(digest),
                "peak_basis": (f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                               f"{sm_max:.0f} MHz (max SM clock)"),
                "ops_per_launch": ops,
                "per_unit": (f"{OPS_INTERACTION} FP32 lane-ops per opponent "
                             f"interaction, {OPS_BALL} per ball evaluation "
                             "(the kernel's own arithmetic)"),
                "survey_count": {
                    "per_unit": (f"{SURVEY_OPS_INTERACTION} per interaction, "
                                 f"{SURVEY_OPS_BALL} per ball evaluation "
                                 "(the plan's estimate before the kernel)"),
                    "ops_per_launch": ops_survey,
                    "achieved": ops_survey / t_launch / 1e12,
                    "frac": ops_survey / t_launch / peak_ops},
                "ncu": ncu,
                "target": ("at least 0.5 of the FP32 pipe: judged on ncu's "
                           "FMA-pipe active fraction (ncu.fma_pipe_active); "
                           "frac and survey_count.frac bracket it by the two "
                           "op counts"),
                "xu": {"achieved": mufu / t_launch / 1e12,
                       "peak": peak_mufu / 1e12, "unit": "T MUFU ops/s",
                       "frac": mufu / t_launch / peak_mufu},
                "kernel_source_digest": digest}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            gs = (float(np.float32(grid.spacing)), grid.nx, grid.ny,
                  float(grid.x0), float(grid.y0))
            r, dt, cores = _cpu_oracle_rate(w, batch, gs, CPU_SAMPLE_STATES)
            r1, dt1, _ = _cpu_oracle_rate(w, batch, gs, 2, cores=1)
            # OpenMP keeps the last thread count: give the later oracle
            # timings all cores again
            _cpu_oracle_rate(w, batch, gs, 1, cores=cores)
            cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": (f"first {CPU_SAMPLE_STATES} states of the "
                              f"batched workload (seed {w.seed}), full grid, "
                              f"all speeds; {dt:.1f} s wall"),
                   "single_thread": {"value": r1, "unit": UNIT, "cores": 1,
                                     "sample": (f"first 2 states, one "
                                                f"thread; {dt1:.1f} s wall")}}
        line = {"metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps,
                "ms_per_step_median": float(np.median(step_ms)),
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _config(w, grid.nx, grid.ny, world),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": int(S * 296),
                        "d2h_bytes_per_step": int(S * 32 + S * words * 4),
                        "ms_per_step": e2e_ms / args.steps},
                "clocks": clk.summary(),
                "gpu_launches": 2 * args.steps,
                "states_per_s": world * S * args.steps / (total_ms / 1e3)}
    searcher.close()
    if rank == 0:
        if world == 1 and not args.no_uneven:
            line["uneven"] = _uneven(args, dev, stream)
        if world == 1 and not args.no_serving:
            line["serving"] = _serving(dev, no_cpu=args.no_cpu_baseline)
        if world == 1 and not args.no_proposal:
            line["proposal"] = _proposal(args, dev, stream)
        if world == 1 and not args.no_dpps:
            line["dpps"] = _dpps(args, dev, stream)
        if world == 1 and not args.no_run:
            line["run_points"] = _run_points(args, dev, stream)
        if world == 1 and not args.no_training:
            line["training"] = _training(args, dev, stream)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _uneven(args, dev, stream):
    """The uneven batch through a batched plan (autotuned, graph-captured):
    8192 states mixing 12x9 m / 11 v 11 and 9x6 m / 6 v 6, grids
    0.025-0.1 m, 1-8 speeds, K 32-128, decel 0.3-0.7; timed like the main
    step (L2 flushed between runs, CUDA events on the plan's stream)."""
    import torch
    from paper_1909_07717_gb300 import pps, synth
    S = args.states or synth.UNEVEN_STATES
    batch = synth.uneven_batch(synth.UNEVEN_SEED, S)
    jobs = pps.jobs_from_batch(batch)
    searcher = pps.Searcher(max_states=S, max_opp=16, device=dev.index,
                            stream=stream)
    plan = pps.Plan(searcher, jobs, S, synth.DEFAULT_PARAMS, autotune=True,
                    graph=True)
    st = searcher.states_to_device(batch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    plan.run(st)             # autotunes and captures the graph
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(2):
        plan.run(st)
    steps = max(3, min(args.steps, 5))
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.run(st)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    best = pps.unpack_best(plan.best.cpu().numpy())
    evals = sum(jobs[i].grid.nx * jobs[i].grid.ny * jobs[i].n_speeds
                * int(batch["n_opp"][i]) for i in range(S))
    groups = [{"opp_slots": g.opp_slots, "speed_slots": g.speed_slots,
               "states": g.n_states, "cta_threads": g.cta_threads,
               "sample_unroll": g.sample_unroll, "items": g.n_items,
               "tuned_ms": [round(float(x), 4) for x in g.tuned_ms]}
              for g in plan.groups()]
    P = np.array([jobs[i].grid.nx * jobs[i].grid.ny for i in range(S)],
                 np.float64)
    V = np.array([jobs[i].n_speeds for i in range(S)], np.float64)
    K = batch["K"].astype(np.float64)
    J = batch["n_opp"].astype(np.float64)
    inter, ball = float((P * K * J).sum()), float((P * K * V).sum())
    props = torch.cuda.get_device_properties(dev)
    roof = _alu_roofline(OPS_INTERACTION * inter + OPS_BALL * ball, ms / 1e3,
                         props.multi_processor_count,
                         f"{OPS_INTERACTION} per opponent interaction "
                         f"(state x point x sample x opponent), {OPS_BALL} "
                         "per ball evaluation (state x point x sample x "
                         "speed), as the single-grid kernel",
                         {"interactions": inter, "ball_evaluations": ball})
    roof["scope"] = "every group's kernels of one graph replay"
    out = {"workload": (f"uneven_{S}: 12x9/11v11 + 9x6/6v6, grids "
                        "0.025-0.1 m, 1-8 speeds, K 32-128 (seed 2)"),
           "value": evals / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
           "states_per_s": S / (ms / 1e3), "first_run_s": first_s,
           "graph": True, "autotuned": True, "groups": groups,
           "roofline": roof,
           "ok": bool(np.all(best["status"] == 0))}
    plan.close()
    searcher.close()
    if not args.no_cpu_baseline:
        # the oracle on 48 states spread over the batch, each on its own
        # grid, one state per host thread at a time
        import oracle
        pick = list(range(0, S, max(1, S // 48)))[:48]
        cores = oracle.max_threads()
        calls, n_evals = [], 0.0

        def call(i):
            g = jobs[i].grid
            gs = (float(np.float32(g.spacing)), g.nx, g.ny,
                  float(np.float32(g.x0)), float(np.float32(g.y0)))
            sp = [float(jobs[i].speeds[v]) for v in range(jobs[i].n_speeds)]
            sub = synth.take(batch, [i])
            return lambda: oracle.search(sub, gs, sp, synth.DEFAULT_PARAMS,
                                         n_threads=1)
        for i in pick:
            calls.append(call(i))
            n_evals += P[i] * V[i] * J[i]
        dt = _oracle_pool_rate(calls, cores)
        oracle.search(synth.take(batch, [0]), (0.5, 2, 2, -6.0, -4.5), [3.0],
                      synth.DEFAULT_PARAMS, n_threads=cores)
        out["cpu_baseline"] = {"value": n_evals / dt, "unit": UNIT,
                               "cores": cores, "kind": "oracle",
                               "sample": (f"{len(pick)} states spread over the "
                                          f"batch, each on its own grid, one "
                                          f"per host thread; {dt:.1f} s wall")}
    return out


def _proposal(args, dev, stream):
    """The learned proposal against the plain search on the same 4096
    held-out states (12x9 m, 8 v 8, K = 64, 4 speeds, 0.025 m grid =
    481x361): one pps_propose (rasterise, predict, top-256 cells, exact
    refinement, full-grid fallback) against one pps_search per batch, both
    timed like the main step; the agreement is the share of states whose
    proposal score is within 2 % of the plain search's."""
    import torch
    from paper_1909_07717_gb300 import pps, synth
    from paper_1909_07717_gb300.proposal import TOPK, Proposal, agreement
    w = synth.PROPOSAL
    S = args.states or w.n_states
    batch = w.states(S)
    pr = Proposal(S, device=dev.index, stream=stream)
    st = pr.searcher.states_to_device(batch)
    exo = pr.searcher.alloc_outputs(S, pr.grid, len(w.speeds), mask=False)
    pro = pr.alloc(S)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps, flush_l2=True):
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            if flush_l2:
                flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    steps = max(3, min(args.steps, 5))
    ms_plain = timed(lambda: pr.exact(st, S, w.speeds, out=exo), steps)
    ms_prop = timed(lambda: pr.run(st, S, w.speeds, out=pro), steps)
    ms_pred = timed(lambda: pr.net.forward(st, S), steps)
    # the stages on their own: the rasteriser (pps_net_raster, which also
    # copies the map out), the tcgen05 network on that map
    # (pps_net_forward_map, which first copies it into the network's
    # 16-channel input)
    maps = torch.empty((S, 46, 61, 8), dtype=torch.int16, device=dev)
    net_out = torch.empty((S, 46, 61), dtype=torch.float32, device=dev)
    ms_raster = timed(lambda: pps.pps_net_raster(pr.net.net, st.data_ptr(), S,
                                                 maps.data_ptr()), steps)
    ms_network = timed(lambda: pps.pps_net_forward_map(
        pr.net.net, maps.data_ptr(), S, 0, net_out.data_ptr()), steps)
    ex = pps.unpack_best(exo["best"].cpu().numpy())
    pb = pps.unpack_best(pro[0].cpu().numpy())
    nofb = pps.unpack_best(pr.run(st, S, w.speeds, fallback=False)[0]
                           .cpu().numpy())
    # small batches (a serving launch holds one or a few frames): latency
    # of each path, no L2 flush, back-to-back calls
    small = {}
    rs = pps.STATE_DTYPE.itemsize
    for m in (1, 16):
        if m > S:
            continue
        sub = st[:m * rs]
        eo = pr.searcher.alloc_outputs(m, pr.grid, len(w.speeds), mask=False)
        po = pr.alloc(m)
        small[str(m)] = {
            "plain_us": 1e3 * timed(lambda: pr.exact(sub, m, w.speeds, out=eo),
                                    10, flush_l2=False),
            "proposal_us": 1e3 * timed(lambda: pr.run(sub, m, w.speeds, out=po),
                                       10, flush_l2=False)}
    pr.close()
    ok = agreement(pb, ex)
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    # network: algorithmic FLOPs of the four 3x3 convolutions on the
    # unpadded channels, no band halo: 2 x 9 x (8x32 + 32x32 + 32x32 + 32x1)
    # per pixel
    flop_px = 2 * 9 * (8 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
    flops = S * 46 * 61 * flop_px
    peak_tc = float(_peaks().get("bf16_tflops", 1920.3)) * 1e12
    net_roof = {"bound": "tensor", "achieved": flops / (ms_network / 1e3) / 1e12,
                "peak": peak_tc / 1e12, "unit": "TFLOP/s (bf16, FP32 accumulate)",
                "frac": flops / (ms_network / 1e3) / peak_tc, "traffic": None,
                "per_unit": f"{flop_px} FLOP per map pixel (unpadded channels, "
                            "no halo)", "flops_per_launch": flops,
                "peak_basis": "measured bf16 cuBLAS burst (MEASURED_PEAKS.json)",
                "ms": ms_network,
                "note": "time includes copying the map into the network's "
                        "16-channel input"}
    # rasteriser: per pixel 4 sub-points x 16 pass-line samples x (8
    # opponent slots x 14 + 4 speeds x 3) FP32 lane-ops of the search's
    # arithmetic (shot angles and the other channels not counted)
    ops_px = 4 * 16 * (8 * OPS_INTERACTION + 4 * OPS_BALL)
    raster_roof = _alu_roofline(S * 46 * 61 * ops_px, ms_raster / 1e3, nsm,
                                f"{ops_px} FP32 lane-ops per map pixel (4 "
                                "sub-points x 16 samples x (8 opponent slots "
                                "x 14 + 4 speeds x 3)); shot angles and the "
                                "other channels not counted",
                                {"pixels": S * 46 * 61})
    raster_roof["ms"] = ms_raster
    roofline = {"network": net_roof, "raster": raster_roof,
                "refine_topk_finalize_ms": ms_prop - ms_pred,
                "shares_of_the_call": {
                    "raster": ms_raster / ms_prop,
                    "network": ms_network / ms_prop,
                    "top-k, refinement, finalize":
                        (ms_prop - ms_pred) / ms_prop}}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        g = pps.fine_grid_12x9()
        gs = (float(np.float32(g.spacing)), g.nx, g.ny, float(g.x0),
              float(g.y0))
        t0 = time.perf_counter()
        oracle.search(synth.take(batch, list(range(4))), gs, w.speeds,
                      w.params)
        dt = time.perf_counter() - t0
        cpu = {"value": 4 / dt, "unit": "states/s",
               "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"the first 4 states, full 0.025 m grid; {dt:.1f} s "
                         "wall (the plain search: the proposal's judge)"}
    return {"workload": f"{w.name} (seed {w.seed}, held out of training)",
            "roofline": roofline, "cpu_baseline": cpu,
            "topk": TOPK, "ms_plain": ms_plain, "ms_proposal": ms_prop,
            "ms_predict": ms_pred,
            "plain_states_per_s": S / (ms_plain / 1e3),
            "proposal_states_per_s": S / (ms_prop / 1e3),
            "speedup": ms_plain / ms_prop,
            "agree_2pct": float(ok.mean()),
            "same_point": float((pb["idx"] == ex["idx"]).mean()),
            "fallback_states": int((nofb["idx"] == -1).sum()),
            "small_batch_latency": small,
            "refined_points_frac": TOPK * 64 / (481 * 361)}


def _dpps(args, dev, stream):
    """The paper's own parameterisation (Sec. 4.2): from the ball holder,
    128 directions x 64 kick powers, 16 receivers and 16 opponents searched
    along every ball path (K = 64), 4096 states per run; timed like the
    main step.  The metric is the paper's unit: SBIP evaluations (one
    robot's interception search for one candidate pass) per second; the
    oracle's rate on the host cores (4 states) beside it."""
    import torch
    from paper_1909_07717_gb300 import pps, synth
    S = args.states or synth.DPPS_STATES
    prm = pps.dparams_from_dict(synth.DPPS_PARAMS)
    batch = synth.dpps_states(synth.DPPS_SEED, S)
    searcher = pps.Searcher(max_states=S, max_opp=16, device=dev.index,
                            stream=stream)
    rec = torch.from_numpy(pps.pack_dstates(batch).view(np.uint8).copy()).to(dev)
    best = torch.empty(S * 48, dtype=torch.uint8, device=dev)
    mask = torch.empty((S, pps.pps_dpps_mask_words(prm)), dtype=torch.int32,
                       device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def run():
        pps.pps_dpps_search(searcher.ctx, rec.data_ptr(), S, prm,
                            best.data_ptr(), mask.data_ptr())

    for _ in range(2):
        run()
    steps = max(3, min(args.steps, 5))
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    b = np.frombuffer(best.cpu().numpy().tobytes(), pps.DBEST_DTYPE)
    # Sec. 4.1 passing powers and Sec. 4.4 shots: 16 queries per state
    Q = 16 * S
    rng = np.random.default_rng(synth.DPPS_SEED)
    pq = np.zeros(Q, pps.PASS_QUERY_DTYPE)
    pq["state"] = np.repeat(np.arange(S), 16)
    pq["receiver"] = np.tile(np.arange(16), S)
    pq["target"] = rng.uniform([-6, -4.5], [6, 4.5], (Q, 2))
    sq = np.zeros(Q, pps.SHOT_QUERY_DTYPE)
    sq["state"] = pq["state"]
    sq["from"] = rng.uniform([-2, -4.5], [6, 4.5], (Q, 2))

    pqd = torch.from_numpy(pq.view(np.uint8).copy()).to(dev)
    sqd = torch.from_numpy(sq.view(np.uint8).copy()).to(dev)
    pout = torch.empty(Q * pps.PASS_POWER_DTYPE.itemsize, dtype=torch.uint8,
                       device=dev)
    sout = torch.empty(Q * pps.SHOT_DTYPE.itemsize, dtype=torch.uint8,
                       device=dev)

    def timed(fn):
        for _ in range(2):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / steps

    ms_pass = timed(lambda: pps.pps_pass_powers(
        searcher.ctx, rec.data_ptr(), S, pqd.data_ptr(), Q, 0.3, prm,
        pout.data_ptr()))
    ms_shot = timed(lambda: pps.pps_shoot(
        searcher.ctx, rec.data_ptr(), S, sqd.data_ptr(), Q, 6.5, 0.1, prm,
        sout.data_ptr()))
    # Algorithmic work: per candidate the teammates' search runs sample by
    # sample up to the first interception (all K when none) and then,
    # for a pass a teammate gets, the opponents' search likewise; a sample is
    # 16 robot interactions and one ball term, plus one sample more for the
    # group that stops (the holder is found again there).  The samples are
    # counted from the debug times of the first 256 states (untimed run).
    sub_n = min(S, 256)
    C = prm.n_dir * prm.n_pow
    dbg = torch.empty((sub_n, C, 3), dtype=torch.float32, device=dev)
    best2 = torch.empty(sub_n * 48, dtype=torch.uint8, device=dev)
    pps.pps_dpps_search(searcher.ctx, rec.data_ptr(), sub_n, prm,
                        best2.data_ptr(), None, dbg.data_ptr())
    torch.cuda.synchronize()
    dd = dbg.cpu().numpy().astype(np.float64)
    searcher.close()
    samples = _dpps_samples(batch, synth.DPPS_PARAMS, dd)
    per_sample_ops = 16 * OPS_INTERACTION + OPS_BALL
    ops = samples / sub_n * S * per_sample_ops
    props = torch.cuda.get_device_properties(dev)
    roof = _alu_roofline(ops, ms / 1e3, props.multi_processor_count,
                         f"{per_sample_ops} FP32 lane-ops per searched sample "
                         f"(16 robots x {OPS_INTERACTION} + a ball term of "
                         f"{OPS_BALL}); samples per decision counted from "
                         "the first 256 states' interception times",
                         {"samples_per_decision": samples / sub_n})
    robots = int(batch["n_team"][0] + batch["n_opp"][0])
    sbip = S * prm.n_dir * prm.n_pow * robots
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sub = {k: (v[:4] if isinstance(v, np.ndarray) else v)
               for k, v in batch.items()}
        t0 = time.perf_counter()
        oracle.dpps_search(sub, prm.n_dir, prm.n_pow,
                           synth.dpps_oracle_params(synth.DPPS_PARAMS))
        cpu = {"decisions_per_s": 4 / (time.perf_counter() - t0),
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": "first 4 states of the workload"}
    return {"workload": (f"dpps_{S}x{prm.n_dir}x{prm.n_pow}: 12x9 m, 16 v 16,"
                         f" K 64, powers 1-6.5 m/s, slide 5/7 (seed "
                         f"{synth.DPPS_SEED})"),
            "unit": "SBIP evals/s", "value": sbip / (ms / 1e3),
            "ms_per_run": ms, "decisions_per_s": S / (ms / 1e3),
            "sbip_per_decision": prm.n_dir * prm.n_pow * robots,
            "feasible_frac": float(b["n_feasible"].mean()
                                   / (prm.n_dir * prm.n_pow)),
            "pass_powers": {"queries": Q, "ms": ms_pass,
                            "queries_per_s": Q / (ms_pass / 1e3)},
            "shots": {"queries": Q, "ms": ms_shot,
                      "queries_per_s": Q / (ms_shot / 1e3)},
            "cpu_baseline": cpu, "roofline": roof,
            "ok": bool(np.all(b["status"] == 0))}


def _dpps_samples(batch, p, dbg):
    """Samples searched by the direction x power kernel for the states of
    dbg (n, n_dir * n_pow, 3: t_team, t_opp, score): for each group, the
    sample of its first interception recovered from the ball's time there
    (all K samples when none), plus the holder's one."""
    n = dbg.shape[0]
    nd, npw = p["n_dir"], p["n_pow"]
    phi = 2 * np.pi * np.arange(nd) / nd
    ux, uy = np.cos(phi)[:, None], np.sin(phi)[:, None]
    v0 = p["v_lo"] + np.arange(npw) * (p["v_hi"] - p["v_lo"]) / max(npw - 1, 1)
    v = p["slide"] * v0[None, :]
    total = 0.0
    for s in range(n):
        a = float(batch["ball_decel"][s])
        bx, by = (float(x) for x in batch["ball"][s])
        hl, hw = batch["field_len"][s] / 2, batch["field_wid"][s] / 2
        K = int(batch["K"][s])
        with np.errstate(divide="ignore", invalid="ignore"):
            edge = np.minimum.reduce([
                np.where(ux > 0, (hl - bx) / ux, np.inf),
                np.where(ux < 0, (-hl - bx) / ux, np.inf),
                np.where(uy > 0, (hw - by) / uy, np.inf),
                np.where(uy < 0, (-hw - by) / uy, np.inf)])
        S = np.minimum(v * v / (2 * a), np.maximum(edge, 0.0))

        def k_of(t):
            tt = np.where(np.isfinite(t), np.minimum(t, v / a), 0.0)
            dist = v * tt - 0.5 * a * tt * tt
            with np.errstate(divide="ignore", invalid="ignore"):
                k = np.clip(np.round(dist / S * K), 1, K)
            return np.where(np.isfinite(t), k + 1, K)   # + the holder's

        tt = dbg[s, :, 0].reshape(nd, npw)
        to = dbg[s, :, 1].reshape(nd, npw)
        got = np.isfinite(tt)
        total += float(k_of(tt).sum() + np.where(got, k_of(to), 0).sum())
    return total


def _run_points(args, dev, stream):
    """Running points (Sec. 5.1-5.2): the attacking half of a 12 x 9 m field
    at 0.1 m (61 x 91 points), every point scored by the five criteria, the
    best point of each of the four zones and the supporters' zones, for
    4096 states with 16 opponents (one or two guards); timed like the main
    step, with and without the dense score output.  The oracle's rate on the
    host cores (512 states) beside it."""
    import torch
    from paper_1909_07717_gb300 import pps, synth
    S = args.states or synth.RUN_STATES
    prm = pps.rparams_from_dict(synth.RUN_PARAMS)
    batch = synth.run_states(synth.RUN_SEED, S)
    nx, ny = pps.pps_run_grid(12.0, 9.0, prm.spacing)
    searcher = pps.Searcher(max_states=S, max_opp=16, device=dev.index,
                            stream=stream)
    rec = torch.from_numpy(pps.pack_dstates(batch).view(np.uint8).copy()).to(dev)
    out = torch.empty(S * pps.RBEST_DTYPE.itemsize, dtype=torch.uint8,
                      device=dev)
    dense = torch.empty((S, nx * ny), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(with_dense):
        def run():
            pps.pps_run_points(searcher.ctx, rec.data_ptr(), S, prm,
                               out.data_ptr(), None,
                               dense.data_ptr() if with_dense else None,
                               nx * ny if with_dense else 0)
        for _ in range(2):
            run()
        steps = max(3, min(args.steps, 5))
        ev = [(torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            run()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    ms = timed(False)
    ms_dense = timed(True)
    r = np.frombuffer(out.cpu().numpy().tobytes(), pps.RBEST_DTYPE)
    searcher.close()
    pts = S * nx * ny
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sub = {k: (v[:512] if isinstance(v, np.ndarray) else v)
               for k, v in batch.items()}
        t0 = time.perf_counter()
        oracle.run_search(sub, synth.run_oracle_params())
        dt = time.perf_counter() - t0
        cpu = {"points_per_s": 512 * nx * ny / dt, "states_per_s": 512 / dt,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": "first 512 states of the workload"}
    # issue-bound: warp instructions per point from the committed ncu
    # summary, against one warp instruction per scheduler and clock
    prof = _profile_kv("run_kernel_4096.txt")
    roof = None
    if "warp_instructions_per_32_points" in prof:
        props = torch.cuda.get_device_properties(dev)
        nsm = props.multi_processor_count
        sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
        ipp = float(prof["warp_instructions_per_32_points"]) / 32
        peak = nsm * 4 * sm_max * 1e6
        ach = pts * ipp / (ms / 1e3)
        roof = {"bound": "issue", "achieved": ach / 1e12, "peak": peak / 1e12,
                "unit": "T warp-instructions/s", "frac": ach / peak,
                "traffic": None,
                "per_unit": f"{ipp * 32:.1f} warp instructions per 32 points "
                            "(ncu, profiles/run_kernel_4096.txt)",
                "peak_basis": f"{nsm} SMs x 4 schedulers x {sm_max:.0f} MHz",
                "ncu_issue_active": float(prof.get("issue_active", "nan"))}
    return {"workload": (f"run_{S}x{nx}x{ny}: 12x9 m attacking half at "
                         f"0.1 m, 16 opponents (seed {synth.RUN_SEED})"),
            "roofline": roof,
            "unit": "points/s", "value": pts / (ms / 1e3), "ms_per_run": ms,
            "states_per_s": S / (ms / 1e3),
            "ms_per_run_dense": ms_dense,
            "dense_gbs": S * nx * ny * 4 / (ms_dense / 1e3) / 1e9,
            "cpu_baseline": cpu,
            "ok": bool(np.all(r["status"] == 0))}


def _training(args, dev, stream):
    """One training step of the proposal network (pps_net_train_step: the
    rasteriser, the forward pass keeping every activation, the loss, the
    backward pass -- input and weight gradients of the four convolutions --
    and the Adam update) on batches of 256 states of the 12 x 9 m workload
    with exact labels, as train_proposal.py runs it; the forward pass of the
    same batch through the training kernels (pps_net_forward_layers) and
    through the tcgen05 inference kernel beside it."""
    import torch
    from paper_1909_07717_gb300 import pps, synth
    B = 256
    batch = synth.ssl_states(100_000, B, K=64)
    net = pps.Net(dev.index, stream, max_batch=B,
                  weights=pps.init_weights(0, zero_output=True))
    rec = torch.from_numpy(pps.pack_states(batch).view(np.uint8).copy()).to(dev)
    rng = np.random.default_rng(0)
    lab = torch.from_numpy(rng.normal(0.3, 0.4, (B, 46, 61))
                           .astype(np.float32)).to(dev)
    out = torch.empty((B, 46, 61), dtype=torch.float32, device=dev)
    steps = 20

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True),
                  torch.cuda.Event(enable_timing=True))
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    step = lambda: pps.pps_net_train_step(  # noqa: E731
        net.net, rec.data_ptr(), lab.data_ptr(), B, 1e-4, want_loss=False)
    pps.pps_net_set_train_kernels(net.net, pps.PPS_NET_TRAIN_MMA_SYNC)
    ms_step_mma = timed(step)
    pps.pps_net_set_train_kernels(net.net, pps.PPS_NET_TRAIN_TCGEN05)
    ms_step = timed(step)
    pps.pps_net_sync(net.net)
    ms_fwd_layers = timed(lambda: pps.pps_net_forward_layers(
        net.net, rec.data_ptr(), B, out.data_ptr()))
    ms_fwd_tc = timed(lambda: pps.pps_net_forward(net.net, rec.data_ptr(), B,
                                                  out.data_ptr()))
    net.close()
    return {"workload": f"train_step_{B}: 12x9 m, 8 v 8, K 64 features",
            "batch": B, "kernels": "tcgen05", "ms_per_step": ms_step,
            "states_per_s": B / (ms_step / 1e3),
            "ms_per_step_mma_sync": ms_step_mma,
            "speedup_over_mma_sync": ms_step_mma / ms_step,
            "ms_forward_training_kernels": ms_fwd_layers,
            "ms_forward_tcgen05": ms_fwd_tc,
            "note": "steps back to back with no L2 flush, as training runs "
                    "them"}


def _serving(dev, seconds=2.0, no_cpu=False):
    """The serving loop: 512 simulated matches at 60 Hz (12x9 or 9x6 fields,
    6-11 opponents, 0.05 m grid, 4 speeds, K = 32) replayed in real time
    through a pps_server (8 streams, continuous batching), once in each
    mode: exact (every frame on its full grid, 128 MiB mask pool) and
    proposal (the serving network ranks the map cells, the exact search
    refines the best 256 and searches the full grid of a frame whose cells
    hold no feasible pass).  Frame latency is arrival -> result on the
    host.  The default mode is the one with the lower p99 at this load; the
    proposal's agreement with the exact results of the same frames is
    reported beside it."""
    from paper_1909_07717_gb300 import pps, synth
    from paper_1909_07717_gb300.proposal import TOPK, agreement
    hz = 60.0
    M, F = synth.SERVING_MATCHES, int(seconds * hz)
    frames = synth.serving_matches(synth.SERVING_SEED, M, F)
    rec = pps.pack_states(frames)
    jobs = pps.match_jobs(frames)
    weights = np.ascontiguousarray(pps.load_net_weights(pps.SERVING_WEIGHTS),
                                   np.float32)
    prm = pps.params_from_dict(synth.DEFAULT_PARAMS)
    modes, results = {}, {}
    for mode in ("exact", "proposal"):
        # 8 streams, each launch enqueued as soon as a stream is free (no
        # gathering window): at this load the lowest latency of the
        # settings measured (4 or 8 streams x 0, 10, 25, 50 us windows)
        if mode == "exact":
            desc = pps.pps_server_desc(dev.index, 8, 512, 65536, 128 << 20,
                                       16, 0, prm)
        else:
            desc = pps.pps_server_desc(dev.index, 8, 512, 65536, 0, 16, 0,
                                       prm, pps.PPS_SERVE_PROPOSAL, TOPK,
                                       weights.ctypes.data)
        srv = pps.pps_server_create(desc)
        try:
            # warm-up: one match's frames back to back
            pps.pps_server_replay(srv, rec[:F], jobs, 1, F, 1e4)
            res = np.zeros(M * F, pps.RESULT_DTYPE)
            st = pps.pps_server_replay(srv, rec, jobs, M, F, hz, res)
        finally:
            pps.pps_server_destroy(srv)
        d = st.as_dict()
        results[mode] = res
        modes[mode] = {
            "frames": int(d["completed"]), "p50_us": d["p50_us"],
            "p99_us": d["p99_us"], "max_us": d["max_us"],
            "mean_us": d["mean_us"], "states_per_s": d["states_per_s"],
            "mean_batch": d["mean_batch"],
            "queue_p50_us": float(np.percentile(res["queue_ns"], 50) / 1e3),
            "queue_p99_us": float(np.percentile(res["queue_ns"], 99) / 1e3),
            "ok": bool(np.all(res["status"] == 0))}
    ok = agreement(results["proposal"]["best"], results["exact"]["best"])
    modes["proposal"]["agree_2pct"] = float(ok.mean())
    modes["proposal"]["topk"] = TOPK
    default = min(modes, key=lambda m: modes[m]["p99_us"])
    out = {"workload": (f"serving_{M}x60Hz: 12x9/9x6, 6-11 opp, grid 0.05 m,"
                        " 4 speeds, K 32 (seed 4)"),
           "default_mode": default, "modes": modes}
    out.update({k: modes[default][k] for k in
                ("frames", "p50_us", "p99_us", "max_us", "mean_us",
                 "states_per_s", "mean_batch", "ok")})
    if not no_cpu:
        # the oracle's full-grid search of a sample of the frames, each on
        # its own grid, on all host cores
        import oracle
        flat = {k: v for k, v in frames.items() if isinstance(v, np.ndarray)}
        pick = list(range(0, M * F, (M * F) // 8))[:8]
        t0 = time.perf_counter()
        for i in pick:
            sub = synth.take(flat, [i])
            g = pps.pps_grid_from_field(float(flat["field_len"][i]),
                                        float(flat["field_wid"][i]),
                                        float(flat["spacing"][i]))
            gs = (float(np.float32(g.spacing)), g.nx, g.ny, float(g.x0),
                  float(g.y0))
            oracle.search(sub, gs, [float(x) for x in
                                    flat["speeds"][i][:int(flat["n_speeds"][i])]],
                          synth.DEFAULT_PARAMS)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(pick) / dt, "unit": "frames/s",
                               "cores": oracle.max_threads(), "kind": "oracle",
                               "sample": f"{len(pick)} frames of the replay, "
                                         f"full grids; {dt:.1f} s wall"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pps", "reference"], default="pps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven-batch plan measurement")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-loop replay")
    ap.add_argument("--no-proposal", action="store_true",
                    help="skip the learned-proposal comparison")
    ap.add_argument("--no-dpps", action="store_true",
                    help="skip the direction x power search")
    ap.add_argument("--no-run", action="store_true",
                    help="skip the running-point search")
    ap.add_argument("--no-training", action="store_true",
                    help="skip the proposal network's training step")
    ap.add_argument("--states", type=int, default=0,
                    help="states per GPU (default: the workload's 4096); "
                         "smaller only for profiling captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_pps(args)


if __name__ == "__main__":
    sys.exit(main())
