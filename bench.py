"""Benchmark of the per-step particle loop (particle-steps/s, HBM roofline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload C5|C2|C1]
                    [--particles P] [--impl b300|reference]

One step = one PIC cycle of the whole line (push with drag, Monte-Carlo RICS
and pairs, move, integer deposit; surface supply; FP64 field update; a cell
sort every sort_every steps).  The default workload is the pair-loaded
r_eq = 30 line with 262,144 cells and 1e9 macroparticles (synthetic state;
the paper publishes no data set).  With torchrun (N > 1) every rank advances
its own independent line (replicas; weak scaling) and the value is the
particle-steps of all ranks over the slowest rank's time.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_17661_b300 import workloads as W  # noqa: E402

BYTES_PER_SLOT = 21      # push: read pos 4 + u 4 + w 4 + sp 1, write pos 4 + u 4
BYTES_PER_DRAW = 8       # id read of a lepton that draws a Philox number
BYTES_PER_CREATED = 21   # pos, u, w, sp, id written per created particle
SORT_BYTES_PER_SLOT = 62 # a sort reads and writes 29 B per slot, plus a 4 B key pass
NOMINAL_HBM_GBS = 7700.0 # B300 HBM3e, nominal

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the default push (the streaming push, k_push_stream) per slot it read, from
# one ncu capture of the same push source on a smaller line at the same
# density (1e8 macroparticles, 26,214 cells: 2.0616 GB for 1.0e8 slots);
# traffic grows in proportion to the slots.  Reported only while the push's
# source -- push_device.h (the per-particle physics) and push_stream.cu (the
# kernel) -- hashes to the captured one, else null.
PUSH_TRAFFIC = {"sources_sha256": "0db06d793185bb8f8d7ac1119b7dcd4cc9ed656666c12bdd8554a450e53fa8dc", "bytes_per_slot": 20.616}
PUSH_SOURCES = ("paper_2609_17661_b300/csrc/push_device.h", "paper_2609_17661_b300/csrc/push_stream.cu")


def _push_sources_sha256():
    import hashlib
    text = ""
    for p in PUSH_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            text += f.read()
    return hashlib.sha256(text.encode()).hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cfg_for(args):
    cfg = W.config(args.workload)
    if args.cells:
        cfg["n_cells"] = args.cells
    if args.workload == "C5":
        cfg["capacity"] = int(args.particles * 1.06) + (1 << 20)
    if args.atmosphere:
        cfg["inject_mode"] = W.INJECT_TOPUP
    if args.annihilate_every:
        cfg["annihilate_every"] = args.annihilate_every
    return cfg


def make_state_pinned(cfg, total):
    """Host state in pinned memory (the e2e leg copies it every run)."""
    import torch
    n = int(W.pair_loaded_counts(cfg["n_cells"], total).sum())
    buf = {"pos": torch.empty(n, dtype=torch.int32, pin_memory=True),
           "u": torch.empty(n, dtype=torch.float32, pin_memory=True),
           "w": torch.empty(n, dtype=torch.float32, pin_memory=True),
           "sp": torch.empty(n, dtype=torch.uint8, pin_memory=True),
           "id": torch.empty(n, dtype=torch.int64, pin_memory=True)}
    view = {"pos": buf["pos"].numpy().view(np.uint32), "u": buf["u"].numpy(), "w": buf["w"].numpy(),
            "sp": buf["sp"].numpy(), "id": buf["id"].numpy().view(np.uint64)}
    W.load_pair_loaded(cfg, total, out=view)
    return buf, view, n


def _oracle_run(cfg, st, budget_s, max_steps, threads):
    """Steps of the oracle on state `st` with `threads` threads until about
    `budget_s` seconds or `max_steps` steps: (particle-steps/s, steps)."""
    import oracle as O
    O.set_threads(threads)
    o = W.to_oracle(st, cfg["n_cells"])
    S = O.Sim(cfg)
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    t0 = time.perf_counter()
    S.step(1)
    t1 = time.perf_counter()
    steps = int(max(1, min(max_steps, budget_s / max(t1 - t0, 1e-9))))
    units = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        units += S.n
        S.step(1)
    dt = time.perf_counter() - t0
    O.set_threads(1)
    return units / dt, steps


def cpu_baseline(cfg, sample_total, budget_s, max_steps):
    """The FP64 oracle, as it stands, on a bounded sample of the workload
    (the same line and physics with about `sample_total` macroparticles in
    the same pair-loaded profile): on every host core (its OpenMP build,
    bit-identical to one thread) and, beside it, on one core."""
    cores = os.cpu_count() or 1
    # enough of the oracle's 4096-particle blocks for every core
    total = int(max(sample_total, 4096 * 4 * cores))
    st = W.load_pair_loaded(cfg, total, seed=7)
    v_all, steps = _oracle_run(cfg, st, budget_s, max_steps, cores)
    v_one, steps1 = _oracle_run(cfg, st, 0.3 * budget_s, max_steps, 1)
    return {"value": v_all, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "single_core_value": v_one,
            "sample": f"{st['pos'].size} macroparticles of the same line and profile, {steps} steps on {cores} "
                      f"threads ({steps1} on one) (the oracle's C, FP64, OpenMP over blocks of particles)"}, \
        steps, st["pos"].size


def tp_cfg():
    """The test-particle map's physics: B*/B_QED = 10, 1 keV radially
    streaming photons, physical drag."""
    return W.config("C1", kT_keV=1.0, photon_model=0, drag_scale=1.0)


def cpu_baseline_tp(r_all, t_max, budget_s):
    """The oracle's test-particle line (single thread, as it stands) on a
    bounded sample of the map's lines, evenly spread in r_eq."""
    import oracle as O
    cfg = tp_cfg()
    idx = np.unique(np.linspace(0, r_all.size - 1, 64).astype(np.int64))
    steps, done = 0.0, 0
    t0 = time.perf_counter()
    for k in idx:
        steps += O.tp_line(cfg, float(r_all[k]), 1000.0, 1e-3, t_max)["steps"]
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": steps / t, "unit": "line-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} of the {r_all.size} lines, evenly spread in r_eq, the same dt and t_max "
                      f"(single-threaded C, FP64)"}, steps, t


def cpu_baseline_ensemble(cfgs, counts, theta, budget_s, per_line=20000):
    """The oracle (single thread, as it stands) on a bounded sample of the
    ensemble: lines spread over the set, `per_line` macroparticles each in
    the same pair-loaded profile, drag law SURROGATE with the network
    `theta`, stepped until the budget is spent."""
    import oracle as O
    idx = np.unique(np.linspace(0, len(cfgs) - 1, 8).astype(np.int64))
    units, done = 0.0, 0
    t_sum = 0.0
    for k in idx:
        st = W.load_pair_loaded(cfgs[k], per_line, seed=7)
        o = W.to_oracle(st, cfgs[k]["n_cells"])
        S = O.Sim(cfgs[k])
        S.set_surrogate(theta)
        S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
        t0 = time.perf_counter()
        S.step(2)
        t_sum += time.perf_counter() - t0
        units += 2 * o["s"].size
        done += 1
        if t_sum > budget_s:
            break
    return {"value": units / t_sum, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} of the {len(cfgs)} lines, {per_line} macroparticles each in the same profile, "
                      f"2 steps, drag law SURROGATE (single-threaded C, FP64)"}, units, t_sum


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in ("TP", "C4"):
        return run_reference_other(args)
    cfg = cfg_for(args)
    sample = args.ref_sample
    cb, steps, n = cpu_baseline(cfg, sample, budget_s=max(5.0, 0.6 * args.steps), max_steps=args.steps)
    v = cb["value"]
    line = {"metric": "particle-steps/s", "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": 1, "ms_per_step": n / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "cells": cfg["n_cells"], "r_eq": cfg["r_eq"],
                       "particles": n, "sort_every": cfg["sort_every"], "drag": "table"},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_other(args):
    """The reference arm of the map and ensemble workloads: the oracle on a
    bounded sample of the same workload."""
    if args.workload == "TP":
        r = np.geomspace(2.0, 100.0, args.tp_lines)
        cb, units, t = cpu_baseline_tp(r, args.tp_tmax, budget_s=max(5.0, 0.6 * args.steps))
        metric, name = "line-steps/s", (f"test-particle drag map, {r.size} dipole lines r_eq in [2, 100], "
                                         f"gamma0 1000, b*=10, 1 keV radial photons, dt 1e-3, t_max {args.tp_tmax:g}")
    else:
        cfgs, counts = W.ensemble_configs()
        cb, units, t = cpu_baseline_ensemble(cfgs, counts, W.sur_init_params(0), budget_s=max(5.0, 0.6 * args.steps))
        metric, name = "particle-steps/s", ("ensemble of 256 dipole lines, r_eq log-uniform in [2, 30], 512-65536 "
                                             "cells affine in arc length, 1e4-1e7 macroparticles each, surrogate drag")
    v = cb["value"]
    line = {"metric": metric, "value": v, "unit": metric, "n_gpus": args.gpus, "steps": args.steps, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name}, "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": v, "unit": metric, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name(args):
    cells = args.cells or 262144
    name = {"C5": f"pair-loaded dipole line r_eq=30, {cells} cells, {args.particles:.3g} macroparticles, "
                  "table drag, pairs on (n_max cap), sort every 20",
            "C2": "dipole line r_eq=20, 65536 cells, 256/cell, surface injection",
            "C1": "dipole line r_eq=4, 1024 cells, 32/cell"}[args.workload]
    if args.atmosphere:
        name += ", atmosphere topped up with gravity"
    if args.annihilate_every:
        name += f", annihilation at n_max every {args.annihilate_every} steps"
    return name


def reduce_over_ranks(elapsed, units, world, device):
    """(max of `elapsed`, sum of `units`) over the ranks of the default
    process group: the whole job's time is its slowest rank's, its work is
    every rank's."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2609_17661_b300 import Line

    cfg = cfg_for(args)
    cfg["seed"] = 1 + rank
    t_gen = time.perf_counter()
    buf, view, n = make_state_pinned(cfg, int(args.particles))
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream()
    line = Line(cfg, stream=stream.cuda_stream)
    line.set_state(view)
    line.sort()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    line.step(args.warmup)
    d0 = line.diag()
    line.timing(True)
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    line.step(args.steps)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    d1 = line.diag()
    line.timing(False)
    units = d1["push_slots"]
    draws = d1["rng_draws"] - d0["rng_draws"]
    created = (d1["pairs_created"] - d0["pairs_created"]) * 2 + (d1["injected"] - d0["injected"])
    ms_max, units_all = reduce_over_ranks(ms, units, world, "cuda")
    value = units_all / (ms_max * 1e-3)

    # roofline of the push kernel: algorithmic bytes per launch / mean launch time
    launches = d1["push_launches"]
    push_bytes = BYTES_PER_SLOT * units + BYTES_PER_DRAW * draws + BYTES_PER_CREATED * created
    peak, peak_kind = _peaks()
    achieved = push_bytes / (d1["push_ms"] * 1e-3) / 1e9
    traffic = None
    variant = d1["push_variant"]
    # the capture is of the default push (variant 0) without the atmosphere
    # (another instantiation)
    if _push_sources_sha256() == PUSH_TRAFFIC["sources_sha256"] and not args.atmosphere and variant == 0:
        traffic = PUSH_TRAFFIC["bytes_per_slot"] * units / max(launches, 1)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_push_stream" if variant in (0, 6, 7) else "k_push",
            "push_variant": variant, "launches": launches,
            "bytes_per_launch": push_bytes / max(launches, 1), "slots_per_launch": units / max(launches, 1),
            "mean_launch_ms": d1["push_ms"] / max(launches, 1),
            "peak_kind": peak_kind, "push_share_of_step": d1["push_ms"] / ms,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    # the whole step against the roofline: push bytes plus the sort's share
    # (read and write every slot with its id, and a key pass, once per
    # sort_every steps), over the step time
    sorts = sum(1 for k in range(d0["step"] + 1, d0["step"] + args.steps + 1) if k % cfg["sort_every"] == 0)
    step_bytes = push_bytes + sorts * SORT_BYTES_PER_SLOT * (units / max(launches, 1))
    roof["step"] = {"achieved": step_bytes / (ms * 1e-3) / 1e9, "frac": step_bytes / (ms * 1e-3) / 1e9 / peak,
                    "bytes_per_particle_step": step_bytes / max(units, 1)}

    # end to end through the C ABI from pinned host buffers: upload the state,
    # K steps, read back the diagnostics and the field every step.  A
    # time-stepper takes its input once: the upload is counted per step
    # (amortised over the K steps) and also reported on its own, beside the
    # host traffic every step has in steady state (diag, E, J)
    e2e = None
    if not args.no_e2e:
        barrier()
        Eh = np.zeros(cfg["n_cells"])
        t0 = time.perf_counter()
        line.set_state(view)
        line.sort()
        t_up = time.perf_counter() - t0
        for _ in range(args.steps):
            line.step(1)
            line.diag()
            line.fields()
        barrier()
        te = time.perf_counter() - t0
        te_max, units_e = reduce_over_ranks(te, args.steps * n, world, "cuda")
        h2d = 21 * n
        d2h_step = 8 * cfg["n_cells"] + 8 * cfg["n_cells"] + 256
        steady_max, _ = reduce_over_ranks(te - t_up, args.steps * n, world, "cuda")
        e2e = {"value": units_e / te_max, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h_step,
               "h2d_bytes_once": h2d, "upload_s": t_up,
               "steady": {"value": units_e / steady_max, "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": d2h_step},
               "note": "the state is uploaded once per run (a resident time-stepper); h2d_bytes_per_step is "
                       "that upload spread over the run's steps, so the figure grows with --steps; 'steady' "
                       "leaves the upload out"}
        del Eh

    line.close()
    sur = None
    if not args.no_surrogate:
        sur = surrogate_leg(cfg, view, stream, args.sur_steps, value / max(world, 1), barrier)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, _, _ = cpu_baseline(cfg, args.cpu_sample, budget_s=15.0, max_steps=500)

    if rank == 0:
        out = {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": workload_name(args), "cells": cfg["n_cells"], "r_eq": cfg["r_eq"],
                          "particles": n, "sort_every": cfg["sort_every"], "drag": "table",
                          "l2": "inputs (21 B x particles) far larger than the 126 MB L2",
                          "parallelism": f"replicas x{world}"},
               "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cb, "surrogate": sur,
               "gpu_launches": gpu_launches(args.steps, cfg, d0["step"]),
               "pairs_created": d1["pairs_created"] - d0["pairs_created"], "rng_draws": draws,
               "branches": {k: d1[k] - d0[k] for k in ("limiter_branch", "newton_branch", "scatters", "psc_clamped",
                                                       "pairs_rejected_nmax", "lost_north", "lost_south")},
               "setup_s": {"host_state": t_gen}}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


SUR_TENSOR_FLOP_PER_ROW = 2 * 2 * 64 * 64   # layers 2 and 3, 2 flop per multiply-add (the tangent doubles it)


def surrogate_leg(cfg, view, stream, steps, value_plain, barrier):
    """The same line and state with drag law SURROGATE: the line's network is
    trained first (1e7 quadrature samples over its own (gamma, s) box, 20
    epochs of 8192, cosine schedule), then `steps` steps are timed like the
    plain path.  (The ensemble workload trains one network for r_eq in
    [2, 30] and reports its accuracy on its own line.)"""
    import torch
    from paper_2609_17661_b300 import Line
    cs = dict(cfg, drag_law=3)
    line = Line(cs, stream=stream.cuda_stream)
    line.sur_set_params(W.sur_init_params(0))
    rep = line.train_surrogate(**W.sur_train_line(cfg["r_eq"]))
    line.set_state(view)
    line.sort()
    line.step(1)
    d0 = line.diag()
    line.timing(True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    line.step(steps)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    d1 = line.diag()
    line.close()
    units = d1["push_slots"]
    rows = d1["sur_rows"] - d0["sur_rows"] + d1["sur_rows_tangent"] - d0["sur_rows_tangent"]
    push_s = d1["push_ms"] * 1e-3
    peak = _bf16_peak()
    tflops = rows * SUR_TENSOR_FLOP_PER_ROW / push_s / 1e12
    v = units / (ms * 1e-3)
    return {"value": v, "unit": "particle-steps/s", "steps": steps, "ms_per_step": ms / steps,
            "vs_plain": v / value_plain, "drag": "surrogate (the line's own network, trained in the run)",
            "network_rows_per_particle_step": (d1["sur_rows"] - d0["sur_rows"]) / max(units, 1),
            "tangent_rows_per_particle_step": (d1["sur_rows_tangent"] - d0["sur_rows_tangent"]) / max(units, 1),
            "tensor": {"bound": "tensor", "achieved": tflops, "peak": peak[0], "unit": "TFLOP/s",
                       "frac": tflops / peak[0], "peak_kind": peak[1],
                       "flop_per_row": SUR_TENSOR_FLOP_PER_ROW},
            "training": {k: rep[k] for k in ("steps", "samples_ms", "train_ms", "loss_last", "val_count",
                                             "drag_err_median", "drag_err_p99", "drag_err_max",
                                             "lnN_err_median", "lnN_err_p99", "lnN_err_max")}}


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured sustained"
    except Exception:
        return 1400.0, "fallback sustained"


def run_ensemble(args):
    """The batched workload: 256 lines (r_eq log-uniform in [2, 30], cells
    affine in arc length over [512, 65536], twist 0.1-1 of j_psi = 28,
    1e4-1e7 macroparticles each), surrogate drag with one network trained in
    the run, schedule from the autotuner, timed over whole captured
    super-steps (80 steps each)."""
    import torch
    import torch.distributed as dist
    from paper_2609_17661_b300 import Ensemble
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # every rank runs an ensemble of its own (lines drawn with a rank-dependent
    # seed): the lines are independent, so there is no data-path collective
    cfgs, counts = W.ensemble_configs(seed=4 + 1000 * rank)
    t0 = time.perf_counter()
    states = [W.load_pair_loaded(c, int(n), seed=100 + k + 1000 * rank) for k, (c, n) in
              enumerate(zip(cfgs, counts))]
    t_gen = time.perf_counter() - t0
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(W.sur_init_params(0))
    rep = ens.lines[0].train_surrogate(**W.SUR_TRAIN_SHARED)
    for ln, st in zip(ens.lines, states):
        ln.set_state(st)
        ln.sort()
    del states
    t0 = time.perf_counter()
    chunk, cad, cost = ens.tune(trial_steps=10)
    t_tune = time.perf_counter() - t0
    ens.step(80)                      # capture and one warm-up replay
    torch.cuda.synchronize()
    slots0 = sum(ln.diag()["n_slots"] for ln in ens.lines)
    rows0 = sum(ln.diag()["sur_rows"] + ln.diag()["sur_rows_tangent"] for ln in ens.lines)
    steps = max(80, (args.steps // 80) * 80)
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    es = ens.stream()            # the ensemble launches on a stream of its own
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(es)
    ens.step(steps)
    e1.record(es)
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    diags = [ln.diag() for ln in ens.lines]
    slots1 = sum(d["n_slots"] for d in diags)
    rows = sum(d["sur_rows"] + d["sur_rows_tangent"] for d in diags) - rows0
    units = 0.5 * (slots0 + slots1) * steps      # slots per step, averaged over the run
    ms_max, units_all = reduce_over_ranks(ms, units, world, "cuda")
    _, rows_all = reduce_over_ranks(ms, rows, world, "cuda")
    _, particles_all = reduce_over_ranks(ms, int(counts.sum()), world, "cuda")
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        ens.close()
        return
    value = units_all / (ms_max * 1e-3)
    peak = _bf16_peak()
    tflops = rows_all * SUR_TENSOR_FLOP_PER_ROW / (ms_max * 1e-3) / 1e12 / world
    out = {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
           "steps": steps, "warmup": 80, "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
           "config": {"workload": "ensemble of 256 dipole lines, r_eq log-uniform in [2, 30], 512-65536 cells "
                                  "affine in arc length, 1e4-1e7 macroparticles each, surrogate drag",
                      "lines": len(cfgs) * world, "particles": int(particles_all),
                      "cells": int(sum(c["n_cells"] for c in cfgs)),
                      "parallelism": "one ensemble of 256 lines per GPU, all lines per launch" if world > 1
                      else "one GPU, all lines per launch",
                      "l2": "inputs far larger than the 126 MB L2"},
           "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak[0], "unit": "TFLOP/s",
                        "frac": tflops / peak[0], "peak_kind": peak[1], "kernel": "k_ens_push (network layers)",
                        "traffic": None},
           "clocks": clocks,
           "autotuner": {"chunk_tiles": {str(k): int((chunk == k).sum()) for k in (1, 4, 16)},
                         "sort_every": {str(k): int((cad == k).sum()) for k in (10, 20, 40)},
                         "tune_s": t_tune},
           "training": {k: rep[k] for k in ("steps", "samples_ms", "train_ms", "drag_err_median", "drag_err_p99",
                                            "lnN_err_median", "lnN_err_p99")},
           "gpu_launches": 4 * steps + sum(7 * (steps // int(c)) for c in cad),
           "cpu_baseline": None if args.no_cpu else
           cpu_baseline_ensemble(cfgs, counts, ens.lines[0].sur_get_params(), budget_s=15.0)[0],
           "setup_s": {"host_state": t_gen}}
    print(json.dumps(out), flush=True)
    ens.close()


# FP64 operations per line-step of the map kernel (adds, multiplies, and two
# per fused multiply-add), counted by ncu on a map of 4096 lines (1084 =
# 7.57e10 operations over 6.23e7 line-steps); used for the kernel's
# arithmetic roofline against the nominal FP64 rate
TP_FP64_PER_STEP = 1084.0
FP64_NOMINAL_TFLOPS = 1.25


def run_tp_map(args):
    """The test-particle drag map: `--tp-lines` dipole lines (65,536 by
    default), r_eq log-spaced in [2, 100], gamma0 = 1000, B*/B_QED = 10,
    1 keV radially streaming photons, dt = 1e-3 R*/c to the equator or
    `--tp-tmax` R*/c; one FP64 thread per line.  Reports line-steps/s and the
    critical radius found."""
    import torch
    from paper_2609_17661_b300 import tp_map
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    cfg = W.config("C1", kT_keV=1.0, photon_model=0, drag_scale=1.0)
    r = np.geomspace(2.0, 100.0, args.tp_lines)
    tp_map(cfg, r[:64], dt=1e-3, t_max=20.0)            # warm-up
    res, ms = tp_map(cfg, r, dt=1e-3, t_max=args.tp_tmax)
    steps = float(res["steps"].sum())
    third = r[res["region"] == 3]
    roof = None
    if TP_FP64_PER_STEP:
        ach = steps * TP_FP64_PER_STEP / (ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s (FP64)",
                "frac": ach / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal", "kernel": "k_tp_map", "traffic": None}
    out = {"metric": "line-steps/s", "value": steps / (ms * 1e-3), "unit": "line-steps/s", "n_gpus": 1,
           "steps": 1, "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"test-particle drag map, {r.size} dipole lines r_eq in [2, 100], gamma0 1000, "
                                  f"b*=10, 1 keV radial photons, dt 1e-3, t_max {args.tp_tmax:g}",
                      "lines": int(r.size)},
           "roofline": roof, "lines_per_s": r.size / (ms * 1e-3),
           "cpu_baseline": None if args.no_cpu else cpu_baseline_tp(r, args.tp_tmax, budget_s=15.0)[0],
           "r_crit": float(third.min()) if third.size else None,
           "regions": {str(k): int((res["region"] == k).sum()) for k in (1, 2, 3)},
           "gpu_launches": 1}
    print(json.dumps(out), flush=True)


def gpu_launches(steps, cfg, step0):
    """Kernels of this library launched in the timed region: per step push,
    field, finalize (+ inject or top-up with surface supply); per sort hist,
    scan reduce, scan top, scan apply, scatter, done; per annihilation pass
    its scan and cell kernels (after a sort, added when off the cadence)."""
    per = 3 + (1 if cfg["inject_mode"] else 0)
    K = cfg.get("annihilate_every", 0)
    steps_run = range(step0 + 1, step0 + steps + 1)
    sorts = sum(1 for s in steps_run if s % cfg["sort_every"] == 0 or (K and s % K == 0))
    passes = sum(1 for s in steps_run if K and s % K == 0)
    return per * steps + 6 * sorts + 2 * passes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="C5", choices=["C5", "C2", "C1", "C4", "TP"])
    ap.add_argument("--particles", type=float, default=1e9)
    ap.add_argument("--cells", type=int, default=0,
                    help="override the line's cell count (smaller lines at the same density for ncu captures)")
    ap.add_argument("--cpu-sample", type=int, default=200000)
    ap.add_argument("--ref-sample", type=int, default=200000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--sur-steps", type=int, default=3)
    ap.add_argument("--tp-lines", type=int, default=65536)
    ap.add_argument("--tp-tmax", type=float, default=200.0)
    ap.add_argument("--atmosphere", action="store_true",
                    help="the line's supply is the paper's atmosphere (inject mode TOPUP, gravity)")
    ap.add_argument("--annihilate-every", type=int, default=0,
                    help="annihilation at n_max every this many steps (0: off)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "b300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "C4":
        run_ensemble(args)
    elif args.workload == "TP":
        run_tp_map(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
