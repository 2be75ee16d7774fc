#!/usr/bin/env python
"""Benchmark: exact DC N-1 topology evaluations per second on the 10000-bus
synthetic workload (15000 branches, 5000 outages x 15000 monitored branches,
4 timesteps, batches of 8192 topologies with up to 6 splits), one MapElites
iteration (propose, split update, fused N-1 sweep, metrics, insert) per step.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own independent search on its own GPU (the
topologies of different ranks are independent; no collective on the data path)
and rank 0 prints one JSON line; with --shared-archive the ranks keep one
archive instead (one all-gather of the step's candidates per step).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import CONFIGS, config_grid, limits_from_flows, random_topologies  # noqa: E402

METRIC = "N-1 topology evals/s (10k-bus)"
UNIT = "evals/s"
# propose, split update, sweep, metrics, 4 insert kernels (+1 pack for the mma.sync sweeps; +2 with lambda_f2:
# the busbar setup and the busbar sweep)
LAUNCHES_PER_STEP = 8


def rank_seed(rank):
    """Search seed of a rank: every rank runs its own independent search."""
    return 1000 + rank


def max_over_ranks(ms, world, device):
    """The largest of the ranks' times (collective over the default group)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank_units, world, steps, max_ms):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return per_rank_units * world * steps / (max_ms / 1000.0)


def workload_desc(cfg, B, n_dslot=0, n_disc=0):
    c = CONFIGS[cfg]
    d = (f"{cfg}: synthetic {c['n_bus']}-bus grid, {c['n_branch']} branches, "
         f"{c['n_outage'] or c['n_branch']} outages x {c['n_branch']} monitored, T={c['T']}, "
         f"batch {B} topologies with <= {c['k_max']} splits")
    if n_dslot:
        d += f" and <= {n_dslot} of {n_disc} branch disconnections"
    return d


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_10128_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.startswith("sweep"):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, cfg):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{cfg}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def oracle_sample(sg, n_topo, n_out, seed, cores):
    """Oracle evaluations of n_topo topologies over n_out sampled outages each,
    spread over `cores` spawned processes; returns (evals/s extrapolated to the
    full outage set, wall seconds, description)."""
    from oracle import dcflow
    topo = random_topologies(sg, n_topo, seed=seed + 999)
    O = sg.outages.size
    rng = np.random.default_rng(seed)
    outs = np.sort(rng.choice(O, min(n_out, O), replace=False))
    t0 = time.perf_counter()
    dcflow.evaluate_many(sg, list(topo), processes=min(cores, n_topo), outages=outs)
    wall = time.perf_counter() - t0
    equiv = n_topo * len(outs) / O
    desc = (f"{n_topo} random topologies x {len(outs)} of {O} outages each on {min(cores, n_topo)} "
            f"processes, extrapolated linearly to the full outage set")
    return equiv / wall, wall, desc


def make_grid(cfg, device, seed, n_disc=0, n_dslot=0):
    from paper_2605_10128_b300 import Grid
    c = CONFIGS[cfg]
    sg = config_grid(cfg, seed=seed, n_disc=n_disc, n_dslot=n_dslot)
    sg = sg.with_limits(np.ones(sg.n_branch))
    t0 = time.perf_counter()
    g = Grid(sg, device=device)
    create_s = time.perf_counter() - t0
    f0 = g.base_flows()
    lim = limits_from_flows(f0[0], c["n_tight"], seed=seed)
    g.set_limits(lim)
    return sg.with_limits(lim), g, create_s


def run_reference(args, rank, world):
    if rank != 0:
        return
    c = CONFIGS[args.config]
    sg = config_grid(args.config, seed=0)
    from oracle import dcflow
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], c["n_tight"], seed=0))
    cores = os.cpu_count() or 1
    P = min(8, cores)
    n_out = args.ref_outages
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(sg, P, 10, 1, cores)
    vals, walls = [], []
    for k in range(args.steps):
        v, w, desc = oracle_sample(sg, P, n_out, 100 + k, cores)
        vals.append(v)
        walls.append(w)
    value = len(vals) / sum(1.0 / v for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(args.config, c["batch"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MIX = ["mix500", "mix2k", "mix5k", "mix10k"]
# a mix where small grids dominate the work: the 500- and 2000-bus grids at
# 8192 topologies each, the 10000-bus grid at 512
MIX_SMALL = {"mix500": 8192, "mix2k": 8192, "mix10k": 512}


def run_mixed(args, prec, pk, pk_kind):
    """Mixed-grid batching: grids of different size, timestep count and batch
    size evaluated as one unit, per-grid launches, one recorded graph of them,
    and the persistent work list (one launch per stage, eager and recorded);
    each grid's sweep tile variant comes from the autotuner (per-grid modes)."""
    import torch
    from paper_2605_10128_b300 import evaluate_multi, _lib
    mix = MIX_SMALL if args.config == "mixsmall" else {n: CONFIGS[n]["batch"] for n in MIX}
    grids, topos, total = [], [], 0
    tune = {}
    for i, (name, B) in enumerate(mix.items()):
        sg, g, _ = make_grid(name, 0, seed=0)
        g.reserve(B)
        tune[name] = g.autotune(min(B, 512), precision=prec)
        topo = torch.from_numpy(random_topologies(sg, B, seed=11 + i)).cuda()
        grids.append(g)
        topos.append(topo)
        total += B
    jobs = list(zip(grids, topos))
    res = {}
    modes = [("per_grid_launches", _lib.MULTI_SEQUENTIAL), ("one_graph", _lib.MULTI_GRAPH)]
    if prec == 0:
        modes += [("persistent", _lib.MULTI_PERSISTENT), ("persistent_graph", _lib.MULTI_PERSISTENT_GRAPH)]
    for label, mode in modes:
        for _ in range(max(1, args.warmup)):
            evaluate_multi(jobs, precision=prec, mode=mode)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            evaluate_multi(jobs, precision=prec, mode=mode)
        e1.record()
        torch.cuda.synchronize()
        res[label] = e0.elapsed_time(e1) / args.steps
    for g in grids:
        g.sync_status()
    best = min(res, key=res.get)
    line = {"metric": f"N-1 topology evals/s (mixed {'/'.join(n[3:] for n in mix)}-bus batch)",
            "value": total / (res[best] / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[best],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "mix: " + ", ".join(workload_desc(n, B) for n, B in mix.items()),
                       "precision": args.precision, "mode": best,
                       "tile_variants": {n: {"chosen": tune[n][0], "ms_per_variant_at_B512": tune[n][1]} for n in mix}},
            "modes": {k: {"value": total / (v / 1000.0), "unit": UNIT, "ms_per_step": v} for k, v in res.items()},
            "gpu_launches": None}
    print(json.dumps(line), flush=True)


def _best(archive):
    fit, _, filled = archive.export()
    return float(fit[filled.astype(bool)].max()) if filled.any() else -np.inf


def time_to_target(g, prec, variants_spec, seeds, iters, train_steps, stop_at_target=False, seed_base=2000):
    """Time to target on the 10000-bus workload: surrogate-screened MapElites
    against plain MapElites (8192 proposals evaluated exactly per iteration),
    same seeds, same precision.  A screened variant "rank:n" proposes n
    candidates per iteration, scores them, evaluates the best-ranked 8192
    exactly (rank "score": by predicted fitness; "gain": by predicted gain over
    the cell's elite, empty cells first), then runs train_steps training
    steps; "rank:n@w" runs plain iterations (whose exact pairs still train
    the surrogate) before screening from iteration w on.  The target of a
    seed is the best fitness its plain run reaches in `iters` iterations;
    each arm's time to target is the wall time of the first iteration whose
    archive holds a fitness at least as good.  Returns (summary, runs)."""
    import torch
    from scipy.stats import spearmanr
    from paper_2605_10128_b300 import Archive, Surrogate, SCREEN_SCORE, SCREEN_CELL_GAIN
    c = CONFIGS["tto10k"]
    B = c["batch"]
    ds, dm = c["archive"]
    sur_kw = dict(hidden=512, n_load=256, replay=262144, minibatch=8192, lr=1e-3)
    variants = []
    for v in variants_spec.split(","):
        mode, rest = v.split(":")
        n, _, w = rest.partition("@")
        variants.append((v, {"score": SCREEN_SCORE, "gain": SCREEN_CELL_GAIN}[mode], int(n), int(w or 0)))
    # warm-up: lazily built device data and every kernel of both arms
    wa = Archive(g, ds, dm)
    ws = Surrogate(g, seed=1, **sur_kw)
    for it in range(2):
        wa.step(1, it, B, precision=prec)
        wa.step_screened(ws, 1, it, variants[0][2], B, rank_by=variants[0][1], precision=prec, train_steps=1)
    torch.cuda.synchronize()
    wa.close()
    ws.close()

    def run_arm(seed, variant, target=None):
        A = Archive(g, ds, dm)
        S = Surrogate(g, seed=seed, **sur_kw) if variant else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        curve = []
        topo_o = torch.empty(B, g.k_max, dtype=torch.int32, device="cuda")
        fit_o = torch.empty(B, dtype=torch.float32, device="cuda")
        for it in range(iters):
            if S is None:
                A.step(seed, it, B, precision=prec)
            elif it < variant[3]:
                # warm start: plain iteration whose exact pairs train the surrogate
                A.step(seed, it, B, precision=prec, topo_out=topo_o, fitness_out=fit_o)
                S.add(topo_o, fit_o)
                S.train(train_steps, want_loss=False)
            else:
                A.step_screened(S, seed, it, variant[2], B, rank_by=variant[1], precision=prec,
                                train_steps=train_steps)
            curve.append((time.perf_counter() - t0, _best(A)))
            if target is not None and curve[-1][1] >= target:
                break
        g.sync_status()
        rho = None
        if S is not None:
            # rank correlation on fresh proposals of the final archive
            prop = A.propose(seed, iters + 1, B)
            sc = S.score(prop).cpu().numpy().astype(np.float64)
            fit = g.evaluate(prop, precision=prec, d_split=ds, d_moved=dm)["fitness"].cpu().numpy()
            ok = np.isfinite(sc) & np.isfinite(fit)
            rho = float(spearmanr(sc[ok], np.log1p(-fit[ok].astype(np.float64))).statistic)
            S.close()
        A.close()
        return curve, rho

    runs = []
    for k in range(seeds):
        seed = seed_base + k
        plain, _ = run_arm(seed, None)
        target = plain[-1][1]
        t_plain = next(t for t, b in plain if b >= target)
        rec = {"seed": seed, "target_fitness": target, "plain_s": t_plain,
               "plain_s_per_iter": plain[-1][0] / iters,
               "plain_best_by_iter": [round(b, 3) for _, b in plain], "screened": {}}
        for v in variants:
            curve, rho = run_arm(seed, v, target if stop_at_target else None)
            hit = [t for t, b in curve if b >= target]
            rec["screened"][v[0]] = {"time_s": hit[0] if hit else None,
                                     "speedup": (t_plain / hit[0]) if hit else None,
                                     "iterations_run": len(curve),
                                     "final_best": curve[-1][1], "s_per_iter": curve[-1][0] / len(curve),
                                     "spearman_rho": rho, "best_by_iter": [round(b, 3) for _, b in curve]}
        runs.append(rec)
    summary = {}
    for v in variants:
        sp = [r["screened"][v[0]]["speedup"] for r in runs]
        reached = sum(x is not None for x in sp)
        rhos = [r["screened"][v[0]]["spearman_rho"] for r in runs]
        summary[v[0]] = {"reached": f"{reached}/{len(runs)}",
                         "median_speedup": float(np.median(sp)) if reached == len(runs) else None,
                         "speedups": sp,
                         "spearman_rho": rhos, "median_spearman_rho": float(np.median(rhos)),
                         "final_best_minus_target": [r["screened"][v[0]]["final_best"] - r["target_fitness"]
                                                     for r in runs]}
    return summary, runs


def run_surrogate(args, prec):
    """The time-to-target comparison (see time_to_target) as its own JSON line,
    every arm's best-fitness curve included."""
    cfg = "tto10k"
    c = CONFIGS[cfg]
    B = c["batch"]
    sg, g, _ = make_grid(cfg, 0, seed=0)
    g.reserve(B)
    g.autotune(512, precision=prec)
    summary, runs = time_to_target(g, prec, args.variants, args.seeds, args.iters, args.train_steps,
                                   args.stop_at_target, seed_base=args.seed_base)
    head = summary[args.variants.split(",")[0]]["median_speedup"]
    line = {"metric": "time-to-target best fitness (10k-bus), surrogate-screened vs plain MapElites",
            "value": head, "unit": "x (plain s / screened s)",
            "n_gpus": 1, "steps": args.iters, "warmup": 2, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(cfg, B), "precision": args.precision,
                       "variants": args.variants, "exact_per_iter": B,
                       "train_steps_per_iter": args.train_steps,
                       "seeds": args.seeds, "seed_base": args.seed_base, "iterations": args.iters,
                       "stop_at_target": args.stop_at_target},
            "summary": summary, "runs": runs, "gpu_launches": None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="tto10k")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "fp16x3", "tf32x3", "bf16x3", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-outages", type=int, default=120)
    ap.add_argument("--sweep-variant", type=int, default=-1,
                    help="fix the sweep tile variant instead of autotuning (4 = tcgen05, TF32X3 only)")
    ap.add_argument("--iters", type=int, default=60, help="--config surrogate: iterations per arm")
    ap.add_argument("--seeds", type=int, default=6, help="--config surrogate: seeds")
    ap.add_argument("--seed-base", type=int, default=2000, help="--config surrogate: first seed")
    ap.add_argument("--variants", default="score:65536@16,score:65536@8",
                    help="--config surrogate: screened variants rank:proposals[@first screened iteration] "
                         "(rank = score or gain)")
    ap.add_argument("--train-steps", type=int, default=8, help="--config surrogate: training steps per iteration")
    ap.add_argument("--stop-at-target", action="store_true",
                    help="--config surrogate: end a screened arm once it reaches its seed's target")
    ap.add_argument("--ttt-seeds", type=int, default=3,
                    help="default line: seeds of the time-to-target comparison (0: leave it out)")
    ap.add_argument("--ttt-iters", type=int, default=100, help="default line: plain iterations that set the target")
    ap.add_argument("--ttt-variant", default="score:65536@16", help="default line: the screened arm")
    ap.add_argument("--dslots", type=int, default=0, help="branch-disconnection slots per genome (0: splits only)")
    ap.add_argument("--ndisc", type=int, default=0, help="disconnection set size (default: a hundredth of the branches)")
    ap.add_argument("--ddisc", type=int, default=3, help="archive extent over opened branches when --dslots > 0")
    ap.add_argument("--crossover", action="store_true", help="Algorithm 3's mutation/crossover split of each batch")
    ap.add_argument("--p-c1", type=float, default=0.5, help="crossover bias toward the first parent")
    ap.add_argument("--fitness", default="workload", choices=["workload", "f1", "f2"],
                    help="f2: lambda_f2, which adds every busbar outage of each topology")
    ap.add_argument("--shared-archive", action="store_true",
                    help="under torchrun: one archive shared by all ranks (one all-gather of the step's "
                         "(genome, fitness, cell) rows, the same insert on every rank) instead of independent searches")
    ap.add_argument("--epoch", type=int, default=0,
                    help="iterations per epoch: export the archive and its worst-20 lists after each (0: never)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2605_10128_b300 import Archive, PREC_BF16, PREC_BF16X3, PREC_FP16X3, PREC_FP32, PREC_TF32X3

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    prec = {"fp32": PREC_FP32, "fp16x3": PREC_FP16X3, "tf32x3": PREC_TF32X3, "bf16x3": PREC_BF16X3,
            "bf16": PREC_BF16}[args.precision]
    if args.config in ("mix", "mixsmall"):
        if rank == 0:
            pk, pk_kind = peaks()
            run_mixed(args, prec, pk, pk_kind)
        return
    if args.config == "surrogate":
        if rank == 0:
            run_surrogate(args, prec)
        return
    c = CONFIGS[args.config]
    B = args.batch or c["batch"]
    ds, dm = c["archive"]
    n_disc = (args.ndisc or -(-c["n_branch"] // 100)) if args.dslots else 0
    dd = args.ddisc if args.dslots else 1
    mut = (0.2, 0.2, 0.5, 0.1, 2.0, 0.25, 0.25, 0.5, 0.0, int(args.crossover), args.p_c1)
    sg, g, create_s = make_grid(args.config, local, seed=0, n_disc=n_disc, n_dslot=args.dslots)
    g.reserve(B)
    # sweep tile variant chosen by the library's autotuner (timed on 512
    # topologies), unless --sweep-variant fixes it
    if args.sweep_variant >= 0:
        g.set_sweep_shape(prec, args.sweep_variant)
        tuned_shape, tuned_ms = args.sweep_variant, None
    else:
        tuned_shape, tuned_ms = g.autotune(min(B, 512), precision=prec)
    A = Archive(g, ds, dm, dd)
    fit_kind = {"workload": 0, "f1": 1, "f2": 2}[args.fitness]
    if fit_kind == 2:
        g.busbar_reference()  # lambda_b of the unsplit topology, for lambda_f2
    seed = rank_seed(rank)
    stream = torch.cuda.current_stream()
    if args.shared_archive:
        # one repertoire for all ranks: each rank's proposals use its own key
        # derived from the shared seed; the step's rows are all-gathered and
        # inserted on every rank
        from paper_2605_10128_b300.shared_archive import SharedArchive
        shared = SharedArchive(A)

        def step(it):
            shared.step(rank_seed(0), it, B, mutation=mut, precision=prec, fitness_kind=fit_kind)
    else:
        def step(it):
            A.step(seed, it, B, mutation=mut, precision=prec, fitness_kind=fit_kind)

    for it in range(args.warmup):
        step(it)
    g.sync_status()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    g.profile(True)
    barrier()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    n_export = 0
    for it in range(args.warmup, args.warmup + args.steps):
        step(it)
        if args.epoch and (it - args.warmup + 1) % args.epoch == 0:
            # end-of-epoch hand-over: archive snapshot + worst-20 N-1 cases of
            # every cell, copied to the host while the next epoch runs
            A.epoch_wait()
            A.epoch_export(k=20, stream=stream)
            n_export += 1
    t1.record(stream)
    barrier()
    A.epoch_wait()
    clk = clocks.stop()
    g.profile(False)
    elapsed_ms = t0.elapsed_time(t1)
    stage_ms, ncalls = g.profile_read()
    g.sync_status()
    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")
    value = job_throughput(B, world, args.steps, elapsed_ms)

    # end to end through the C ABI: pinned host topologies in, fitness out
    topo_h = torch.from_numpy(random_topologies(sg, B, seed=77 + rank)).pin_memory()
    fit_h = torch.empty(B, dtype=torch.float32).pin_memory()
    topo_d = torch.empty_like(topo_h, device="cuda")
    out = None
    for _ in range(2):
        topo_d.copy_(topo_h, non_blocking=True)
        out = g.evaluate(topo_d, precision=prec, fitness_kind=fit_kind, d_split=ds, d_moved=dm, d_disc=dd,
                         out=out)
        fit_h.copy_(out["fitness"], non_blocking=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        topo_d.copy_(topo_h, non_blocking=True)
        out = g.evaluate(topo_d, precision=prec, fitness_kind=fit_kind, d_split=ds, d_moved=dm, d_disc=dd,
                         out=out)
        fit_h.copy_(out["fitness"], non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, "cuda")
    e2e = job_throughput(B, world, args.steps, e2e_ms)

    # worst-k N-1 export of the archive's elites, the per-epoch hand-over to AC
    # validation (Sec. "AC-Validator", k = 20); timed on its own, outside the steps
    _, gen_a, filled_a = A.export()
    elites = torch.tensor(gen_a[filled_a.astype(bool)], dtype=torch.int32, device="cuda")
    wk = None
    if elites.shape[0] > 0:
        g.worst_k(elites, k=20)
        g.sync_status()
        w0 = torch.cuda.Event(enable_timing=True)
        w1 = torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        g.worst_k(elites, k=20)
        w1.record(stream)
        torch.cuda.synchronize()
        wk_ms = w0.elapsed_time(w1)
        wk = {"topologies": int(elites.shape[0]), "k": 20, "ms": wk_ms,
              "ms_per_topology": wk_ms / int(elites.shape[0])}

    # time to target, surrogate-screened against plain MapElites, on this grid
    # (one GPU: the comparison is per search, not per job)
    ttt = None
    if world == 1 and args.config == "tto10k" and args.ttt_seeds > 0 and not args.dslots and fit_kind == 0:
        t_ttt = time.perf_counter()
        summary, runs = time_to_target(g, prec, args.ttt_variant, args.ttt_seeds, args.ttt_iters, args.train_steps,
                                       stop_at_target=True)
        s_v = summary[args.ttt_variant]
        ttt = {"variant": args.ttt_variant, "seeds": args.ttt_seeds, "target": f"plain best after {args.ttt_iters} "
               "iterations", "reached": s_v["reached"], "median_speedup": s_v["median_speedup"],
               "speedups": s_v["speedups"], "spearman_rho": s_v["spearman_rho"],
               "plain_s": [r["plain_s"] for r in runs],
               "screened_s": [r["screened"][args.ttt_variant]["time_s"] for r in runs],
               "wall_s": round(time.perf_counter() - t_ttt, 1)}

    if rank == 0:
        pk, pk_kind = peaks()
        props = torch.cuda.get_device_properties(local)
        sms = props.multi_processor_count
        sm_mhz = float(pk.get("sm_max_mhz", 2032.0))
        sweep_ms = stage_ms[1] / max(ncalls, 1)
        T = c["T"]
        E_mon = c["n_branch"]
        O = c["n_outage"] or c["n_branch"]
        instr = 2.0 * B * T * E_mon * O  # one FMA + one |.|-max per (topology, t, l, c)
        achieved = instr / (sweep_ms / 1000.0) / 1e12
        peak = sms * 128 * sm_mhz * 1e6 / 1e12
        kname = ("sweep_fp32" if prec == PREC_FP32 else
                 ("sweep_umma" if prec == PREC_TF32X3 and tuned_shape == 4 else "sweep_tc"))
        traffic = ncu_traffic(kname, args.config)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            P = min(8, cores)
            v, w, desc = oracle_sample(sg, P, args.ref_outages, 5, cores)
            cpu = {"value": v, "unit": UNIT, "cores": P, "kind": "oracle", "sample": desc}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(args.config, B, args.dslots, n_disc), "batch": B, "timesteps": T,
                       "precision": args.precision, "parallelism": (f"shared archive x{world} (all-gather per step)" if args.shared_archive
                                       else f"independent searches x{world}"),
                       "l2": "inputs larger than L2 (N tile 305 MB + per-batch workspace ~8 GB)",
                       "step": "one MapElites iteration: propose, exact N-1 evaluation, insert",
                       "fitness": args.fitness,
                       "genome": {"split_slots": c["k_max"], "disconnection_slots": args.dslots,
                                  "disconnection_set": n_disc, "archive": [ds, dm, dd],
                                  "crossover": bool(args.crossover), "p_c1": args.p_c1},
                       "grid_create_s": round(create_s, 2),
                       "sweep_variant": {"chosen": tuned_shape, "ms_per_variant_at_B512": tuned_ms}},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"N-1 sweep ({kname}, variant {tuned_shape})", "sweep_ms_per_launch": sweep_ms,
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({pk_kind} SM max clock)"},
            "pair_rate": {"value": B * world * T * E_mon * O * args.steps / (elapsed_ms / 1000.0),
                          "unit": "(topology, t, monitored branch, outage) pairs/s"},
            "stage_ms_per_step": {"split_update": stage_ms[0] / max(ncalls, 1), "sweep": sweep_ms,
                                  "metrics": stage_ms[2] / max(ncalls, 1),
                                  "busbar_sweep": stage_ms[3] / max(ncalls, 1)},
            "worst_k_export": wk,
            "time_to_target": ttt,
            "epoch_export": ({"every_steps": args.epoch, "exports_in_timed_region": n_export, "k": 20,
                              "cells": A.cells} if args.epoch else None),
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(B * g.genome_width * 4),
                    "d2h_bytes_per_step": int(B * 4)},
            # the mma.sync sweeps repack U, V and g in a launch of their own; for the
            # tcgen05 sweep (variant 4) the split update writes its operand layouts
            "gpu_launches": (LAUNCHES_PER_STEP + (0 if prec == PREC_FP32 or tuned_shape == 4 else 1)
                             + (2 if args.fitness == "f2" else 0)) * args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
