#!/usr/bin/env python
"""Benchmark of the dLouvain-Delta-s time-step update on GB300.

Metric: ms per time-step update (batch sort-merge into G_t + Delta-screening +
multi-level local moving over R_t + compaction), with local-move GTEPS beside
it.  Workload: the LFR-style power-law temporal graph shaped like the paper's
largest run (2,000,000 vertices, 63M temporal edges over 12 time steps,
degree exponent 2.5, community-size exponent 1.5, mixing 0.3, 5 % community
drift and 2 % deletions per step), generated from a fixed seed: exactly the
configuration's 12 steps.  Step 1 is the static start (untimed); W warm-up
steps follow (t = 2..W+1), then K timed steps: t = W+2..12, and when K is
larger than that, the same steps again from a checkpoint of the state after
the warm-up (dcd_save / dcd_load, untimed) until K steps are timed.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

LFR_N = 2_000_000
LFR_EVENTS = 63_000_000
LFR_STEPS = 12
METRIC = "ms per time-step update"
BYTES_PER_ENTRY = 12   # int32 col + int32 weight + int32 neighbour label, per directed entry visited
BYTES_PER_VERTEX = 40  # row_ptr pair, k, label, a_C, |C|, proposal, list entry per active vertex
# DRAM bytes per algorithmic byte of the local-move kernels: 525.9 MB of
# dram__bytes_read.sum + dram__bytes_write.sum over 433.7 MB algorithmic, from
# the ncu capture of one evaluation of every vertex of the n = 1,000,000
# stream at t = 7 (the caches cold, as ncu leaves them before each pass)
LM_TRAFFIC_RATIO = 525.9 / 433.7
LM_KERNELS = ["lm_seg<8,2> (degree <= 16)", "lm_seg<16,2> (<= 32)", "lm_seg<16,4> (<= 64)",
              "lm_seg<32,4> (<= 128)", "lm_seg<32,8> (<= 256)", "lm_cta<128,4> (<= 512)",
              "lm_cta<256,4> (<= 1024)", "lm_cta<512,4> (<= 2048)", "lm_cta<512,8> (<= 4096)",
              "hub_agg + hub_gain + hub_pick + hub_clear (> 4096)"]


def level0_bytes(st):
    """Algorithmic bytes the level-0 local-move kernels read in one update:
    every pass's active entries and vertices, less the first pass's rows whose
    proposals the screening supplied."""
    return (BYTES_PER_ENTRY * (st.edges_level0 - st.edges_level0_screen)
            + BYTES_PER_VERTEX * (st.verts_level0 - st.verts_level0_screen))


def kernel_rows(rows, peak):
    """Per-kernel roofline rows from dcd_eval_bins: algorithmic bytes of one
    evaluation of the bin over its isolated CUDA-event time."""
    out = []
    for var, nv, ne, ms in rows:
        if nv == 0:
            continue
        by = BYTES_PER_ENTRY * ne + BYTES_PER_VERTEX * nv
        gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else None
        out.append({"kernel": LM_KERNELS[var], "vertices": nv, "entries": ne, "ms": ms, "bytes": by,
                    "gbs": gbs, "frac": (gbs / peak) if gbs else None})
    return out


def workload_desc(n: int = LFR_N) -> str:
    return (f"lfr_2m: LFR-style temporal graph, n={n:,}, {int(round(LFR_EVENTS * n / LFR_N)):,} edge events over "
            f"12 time steps by uniform timestamps, degree exponent 2.5 on [20,20000], community-size exponent "
            f"1.5 on [100,50000], mixing mu=0.3, 5% of vertices drift per step, repeated edges accumulate as "
            f"int32 weights, 2% of the previous step's edges deleted")


def make_stream(n: int, T: int = LFR_STEPS, replica: int = 0):
    """The LFR-style stream of the configuration at n vertices (events scaled
    by n / 2,000,000): T = 12 gives the configuration's 12 steps exactly."""
    from paper_1904_08553_gb300 import synth

    synth.build()
    events = int(round(LFR_EVENTS / LFR_STEPS * T * n / LFR_N))
    return synth.lfr(synth.seed_for(1, replica), n, events, T, kmax=min(20_000.0, n / 2),
                     smax=min(50_000.0, n / 4))


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # let the sampler start up (NVML initialisation) before the timed region
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 5.0:
            if Path(self.path).stat().st_size > 0:
                break
            time.sleep(0.05)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

def oracle_steps(stream, first: int, count: int):
    """The oracle (single thread) on the configuration's own stream: step 1
    (the static start, untimed) and the steps before `first` build the state;
    each sample then copies that state (untimed) and times step `first + 1`
    on the copy.  Returns the per-sample seconds, the graph size after the
    timed step and the static step's seconds."""
    import oracle

    oracle.build()
    n = stream.n
    ctx = oracle.Context(n)
    a = time.perf_counter()
    ctx.apply_batch(*stream.steps[0])
    ctx.update(oracle.DELTA)
    s_static = time.perf_counter() - a
    for t in range(1, first):
        ctx.apply_batch(*stream.steps[t])
        ctx.update(oracle.DELTA)
    secs, nnz = [], 0
    for _ in range(count):
        c = ctx.clone()
        a = time.perf_counter()
        c.apply_batch(*stream.steps[first])
        _, _, st = c.update(oracle.DELTA)
        secs.append(time.perf_counter() - a)
        nnz = st.nnz
        del c
    return secs, nnz, s_static


def cpu_baseline(stream, gpu_nnz_mean: float):
    """One measured oracle step of the configuration (step 2, its first
    Delta-screening step, at the full n), beside an nnz-scaled estimate for
    the steps the GPU arm times."""
    secs, nnz, s_static = oracle_steps(stream, 1, 1)
    ms = secs[0] * 1e3
    est = ms * gpu_nnz_mean / max(nnz, 1)
    return {
        "value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
        "sample": (f"oracle (1 thread of {os.cpu_count()} host cores) on the configuration's own stream at "
                   f"n={stream.n:,}: step 2 (the first Delta-screening step, {nnz:,} directed entries) measured "
                   f"once after the static step 1 ({s_static:.1f} s, untimed); the GPU arm's timed steps hold "
                   f"{gpu_nnz_mean:,.0f} entries on average, so scaled by size the oracle would need about "
                   f"{est:,.0f} ms for one of them (an estimate, not measured)"),
        "measured_step": 2, "measured_nnz": int(nnz), "static_step_s": s_static,
        "nnz_scaled_estimate_ms": est,
    }


def reference_arm(args):
    """The oracle as the reference arm: every step is a measured oracle step 2
    of the configuration's stream, started from a copy of the state after
    step 1 (the copy is untimed); W untimed steps, then K timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    stream = make_stream(args.n, LFR_STEPS)
    secs, nnz, s_static = oracle_steps(stream, 1, args.warmup + args.steps)
    timed = secs[args.warmup:]
    v = float(np.mean(timed)) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "higher_is_better": False,
        "n_gpus": args.gpus, "steps": len(timed), "warmup": args.warmup, "ms_per_step": v,
        "dtype": "int64", "data": "synthetic (seeded LFR-style generator)", "scaling": "weak", "vs_baseline": None,
        "config": config_of(args.n),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": (f"oracle (1 thread of {os.cpu_count()} host cores) on the configuration's own "
                                    f"stream at n={args.n:,}: each step is step 2 (the first Delta-screening step, "
                                    f"{nnz:,} directed entries) from a copy of the state after the static step 1 "
                                    f"({s_static:.1f} s, untimed)")},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def config_of(n: int) -> dict:
    return {"workload": workload_desc(n), "mode": "delta",
            "l2": "inputs larger than L2 (G_t holds 50M-126M directed entries, 0.4-1.0 GB, at n=2,000,000)"}


def timed_schedule(warmup: int, steps: int):
    """Step indices (0-based) of the timed steps: the configuration's steps
    after step 1 and the warm-up, replayed from a checkpoint of the state
    after the warm-up until `steps` steps are timed."""
    first = 1 + warmup
    avail = LFR_STEPS - first
    segs, done = [], 0
    while done < steps:
        k = min(avail, steps - done)
        segs.append(list(range(first, first + k)))
        done += k
    return segs


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1904_08553_gb300 import dcd, shard

    stream = make_stream(args.n, LFR_STEPS, replica=rank)
    n = stream.n
    segs = timed_schedule(args.warmup, args.steps)
    dev = torch.device("cuda", local)
    d_ins, d_del = [], []
    for ins, dels in stream.steps:
        d_ins.append(torch.from_numpy(np.ascontiguousarray(ins)).to(dev))
        dd = np.zeros((len(dels), 3), np.int32)
        dd[:, :2] = dels
        d_del.append(torch.from_numpy(dd).to(dev))
    torch.cuda.synchronize()
    ts = torch.cuda.current_stream(dev)
    tmpdir = tempfile.mkdtemp(prefix="dcd_bench_")
    ckpt = os.path.join(tmpdir, "after_warmup.ckpt")

    def run(ctx, t, host=False, lab_host=None):
        ins, dels = stream.steps[t]
        if host:
            ctx.apply_batch(pinned[t][0], pinned[t][1])
            return ctx.update(labels_out=lab_host)
        ctx.apply_batch_device(d_ins[t], len(ins), d_del[t], len(dels))
        return ctx.update(labels_out=None)

    # device memory for the stream's largest graph and batch, reserved once
    # (untimed), so that no update waits on a buffer growing
    nnz_max = 2 * sum(len(i) for i, _ in stream.steps)
    rec_max = max(len(i) + len(d) for i, d in stream.steps)

    # ---- device-resident inputs ----
    ctx = dcd.Context(n, mode=dcd.MODE_DELTA, stream=ts, pass_loop_host=args.pass_loop == "host")
    ctx.reserve(nnz_max, rec_max)
    tune_after = min(max(args.autotune_at, 1), 1 + args.warmup)
    for t in range(0, 1 + args.warmup):
        run(ctx, t)
        if t + 1 == tune_after and not args.no_autotune:
            ctx.autotune(reps=3)  # degree-bin plan for this graph (untimed)
    plan = ctx.bins()
    if len(segs) > 1:
        ctx.save(ckpt)
    stats, total_ms, launches = [], 0.0, 0
    with ClockSampler(local) as clk:
        for si, seg in enumerate(segs):
            if si > 0:  # the state after the warm-up again (untimed)
                ctx.close()
                ctx = dcd.Context.load(ckpt, stream=ts)
                ctx.reserve(nnz_max, rec_max)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            l0 = dcd.dcd_kernel_launches()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ts)
            for t in seg:
                _, q, st = run(ctx, t)
                stats.append(st)
            e1.record(ts)
            torch.cuda.synchronize()
            launches += dcd.dcd_kernel_launches() - l0
            total_ms += e0.elapsed_time(e1)
    total_ms = shard.max_over_ranks(total_ms, device=dev)
    clocks = clk.summary()
    # each degree bin's kernels alone on the last state (untimed): the
    # per-kernel figures that the side-by-side bins of a pass overlap
    kernels = kernel_rows(ctx.eval_bins(reps=3), peaks()[0])
    ctx.close()

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        pinned = []
        for ins, dels in stream.steps:
            pi = torch.from_numpy(np.ascontiguousarray(ins)).pin_memory().numpy()
            # deletes as full dcd_edge records (w unused), so the binding passes
            # the pinned buffer through without a conversion copy
            d3 = np.zeros((len(dels), 3), np.int32)
            d3[:, :2] = dels
            pd = torch.from_numpy(d3).pin_memory().numpy()
            pinned.append((pi, pd))
        lab_host = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
        ctx = dcd.Context(n, mode=dcd.MODE_DELTA, stream=ts)
        ctx.reserve(nnz_max, rec_max)
        ctx.set_bins(*plan)
        for t in range(0, 1 + args.warmup):
            run(ctx, t, host=True, lab_host=lab_host)
        torch.cuda.synchronize()
        h2d, e2e_ms = 0, 0.0
        for si, seg in enumerate(segs):
            if si > 0:  # same state as the device-resident leg after its warm-up
                ctx.close()
                ctx = dcd.Context.load(ckpt, stream=ts)
                ctx.reserve(nnz_max, rec_max)
                torch.cuda.synchronize()
            a = time.perf_counter()
            for t in seg:
                run(ctx, t, host=True, lab_host=lab_host)
                h2d += pinned[t][0].nbytes + pinned[t][1].nbytes
            torch.cuda.synchronize()
            e2e_ms += (time.perf_counter() - a) * 1e3
        e2e_ms = shard.max_over_ranks(e2e_ms / args.steps, device=dev)
        ctx.close()
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d / args.steps),
               "d2h_bytes_per_step": int(n * 4)}
    if os.path.exists(ckpt):
        os.unlink(ckpt)
    os.rmdir(tmpdir)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    ms_step = total_ms / args.steps
    lm_ms = sum(s.ms_local_move for s in stats)
    # entries and vertices the local-move kernels evaluated: the first level-0
    # pass takes the screening's proposals for the sources it summed
    edges = sum(s.edges_scanned - s.edges_level0_screen for s in stats)
    verts = sum(s.verts_scanned - s.verts_level0_screen for s in stats)
    passes = sum(s.iters_total for s in stats)
    gteps = edges / (lm_ms * 1e-3) / 1e9 if lm_ms > 0 else None
    peak, peak_kind = peaks()
    lm_bytes = BYTES_PER_ENTRY * edges + BYTES_PER_VERTEX * verts
    pass_gbs = lm_bytes / (lm_ms * 1e-3) / 1e9 if lm_ms > 0 else None
    # level 0 (the R_t level, where the graph is the full G_t) is the
    # dominant part of the local move; the upper levels are graphs of a few
    # hundred vertices whose passes are launch-bound
    lm0_ms = sum(s.ms_local_move0 for s in stats)
    lm0_bytes = sum(level0_bytes(s) for s in stats)
    l0_gbs = lm0_bytes / (lm0_ms * 1e-3) / 1e9 if lm0_ms > 0 else None
    passes0 = sum(s.iters_level0 for s in stats)
    # per degree-bin kernel class: its share of the algorithmic bytes (the
    # bins of a pass run side by side inside one graph launch, so their times
    # are not separated)
    names = ["lm_seg (degree <= 32)", "lm_seg (33..256)", "lm_cta (257..4096)",
             "hub_agg + hub_gain + hub_pick (> 4096)"]
    bins = []
    for b in range(4):
        by_b = sum(BYTES_PER_ENTRY * st.edges_bin[b] + BYTES_PER_VERTEX * st.verts_bin[b] for st in stats)
        bins.append({"kernel": names[b], "bytes": by_b, "share": by_b / lm_bytes if lm_bytes else None})
    achieved = l0_gbs
    nnz_mean = float(np.mean([s.nnz for s in stats]))
    cpu = cpu_baseline(stream, nnz_mean) if (world == 1 and not args.no_cpu) else None
    cfg = config_of(n)
    if args.pass_loop == "host":
        cfg["pass_loop"] = "host (each local-move pass enqueued by the host)"
    cfg.update({"parallelism": "replicas" if world > 1 else "1 GPU",
                "timed_steps": (f"t={segs[0][0] + 1}..{segs[0][-1] + 1} of 12"
                                + (f", replayed {len(segs)} times from a checkpoint of the state after the warm-up "
                                   f"(the reload is untimed)" if len(segs) > 1 else "")),
                "bin_plan": {"variants": plan[0], "max_degree": plan[1]}})
    line = {
        "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded LFR-style generator)",
        "config": cfg,
        "local_move_gteps": gteps,
        "steps_detail": {
            "r_fraction": float(np.mean([s.r_size / s.n for s in stats])),
            "q_last": stats[-1].q, "nnz_mean": nnz_mean, "nnz_last": stats[-1].nnz,
            "communities_last": stats[-1].communities,
            "ms_merge": float(np.mean([s.ms_merge for s in stats])),
            "ms_screen": float(np.mean([s.ms_screen for s in stats])),
            "ms_local_move": float(np.mean([s.ms_local_move for s in stats])),
            "ms_apply": float(np.mean([s.ms_apply for s in stats])),
            "ms_coarsen": float(np.mean([s.ms_coarsen for s in stats])),
            "coarse0_delta_steps": int(sum(s.coarse0_delta for s in stats)),
            "coarse0_entries_mean": float(np.mean([s.coarse0_entries for s in stats])),
            "ms_finish": float(np.mean([s.ms_finish for s in stats])),
            "passes_per_step": passes / len(stats),
            "passes_level0_per_step": passes0 / len(stats),
            "first_pass_from_screening": float(np.mean([
                s.verts_level0_screen / (s.verts_level0 / s.iters_level0) if s.iters_level0 and s.verts_level0 else 0.0
                for s in stats])),
            "ms_local_move_level0": lm0_ms / len(stats),
            "levels": float(np.mean([s.levels for s in stats])),
        },
        "roofline": {
            "kernel": "level-0 local-move evaluation: the degree-bin kernels of a pass (lm_seg, lm_cta, hub_*) over "
                      "R_t on G_t, run side by side",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": LM_TRAFFIC_RATIO * lm0_bytes / max(passes0, 1),
            "traffic_note": ("DRAM bytes of one level-0 evaluation: its algorithmic bytes x 1.21, the "
                             "DRAM-to-algorithmic ratio of an ncu capture of the same kernels at n = 1,000,000 "
                             "(cold L2, an upper bound for a pass of the timed loop)"),
            "peak_kind": peak_kind,
            "algorithmic_bytes": f"{BYTES_PER_ENTRY} B x entries scanned + {BYTES_PER_VERTEX} B x vertices evaluated",
            "level0_bytes_per_pass": lm0_bytes / max(passes0, 1),
            "all_levels_gbs": pass_gbs,
            "all_levels_frac": (pass_gbs / peak) if pass_gbs else None,
            "bins": bins,
            "kernels_alone": kernels,
            "kernels_alone_note": ("each bin's kernels timed alone (dcd_eval_bins, CUDA events, mean of 3) "
                                   "on the last timed state, evaluating every vertex of positive degree"),
        },
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if world == 1 and not args.no_extra:
        del d_ins, d_del
        torch.cuda.empty_cache()
        line["extra"] = extra_legs(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def extra_legs(args) -> dict:
    """The configuration's other workloads, each timed with CUDA events and
    its own clock record, reported beside the main line: R-MAT scale 24, the
    512-graph batched form, and the learned screen."""
    out = {}
    for name, leg in (("rmat24", rmat_leg), ("batched", batched_leg), ("learned", learned_leg)):
        t0 = time.time()
        try:
            out[name] = leg(args)
        except Exception as e:  # a failing leg is reported, the main line stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.time() - t0
    return out


# ------------------------------------------------------------------ R-MAT scale 24

RMAT_SCALE = 24


def rmat_leg(args):
    """Plain dLouvain-Delta-s on R-MAT scale 24 (16.8M vertices, a=0.57,
    b=c=0.19, edge factor 16, weights 1..8), 12 steps of 1% inserts and 0.5%
    deletes: step 1 static (untimed), then W warm-up steps and the remaining
    steps timed with CUDA events on the context stream (2m >= 2^31 here, so
    the 128-bit gain path runs)."""
    import torch

    from paper_1904_08553_gb300 import dcd, synth

    t0 = time.time()
    stream = synth.rmat(synth.seed_for(2, 0), scale=args.rmat_scale, edge_factor=16, steps=LFR_STEPS,
                        ins_frac=0.01, del_frac=0.005)
    gen_s = time.time() - t0
    n = stream.n
    dev = torch.device("cuda", 0)
    ts = torch.cuda.current_stream(dev)
    ctx = dcd.Context(n, mode=dcd.MODE_DELTA, stream=ts)
    first = 1 + min(args.warmup, LFR_STEPS - 2)
    stats, ms = [], 0.0
    with ClockSampler(0) as clk:
        for t in range(LFR_STEPS):
            ins, dels = stream.steps[t]
            di = torch.from_numpy(np.ascontiguousarray(ins)).to(dev)
            dd = np.zeros((len(dels), 3), np.int32)
            dd[:, :2] = dels
            dd = torch.from_numpy(dd).to(dev)
            torch.cuda.synchronize()
            ctx.apply_batch_device(di, len(ins), dd, len(dels))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ts)
            _, q, st = ctx.update(labels_out=None)
            e1.record(ts)
            torch.cuda.synchronize()
            if t == 0:
                ctx.autotune(reps=2)
            if t >= first:
                stats.append(st)
                ms += e0.elapsed_time(e1)
            del di, dd
    ctx.close()
    peak, peak_kind = peaks()
    lm0_ms = sum(s.ms_local_move0 for s in stats)
    lm0_bytes = sum(level0_bytes(s) for s in stats)
    gbs = lm0_bytes / (lm0_ms * 1e-3) / 1e9 if lm0_ms > 0 else None
    return {
        "workload": (f"rmat{args.rmat_scale}: R-MAT scale {args.rmat_scale} ({n:,} vertices, a=0.57 b=c=0.19), "
                     f"edge factor 16, weights 1..8, 12 steps of 1% inserts and 0.5% deletes"),
        "ms_per_step": ms / len(stats), "timed_steps": f"t={first + 1}..12", "generation_s": gen_s,
        "r_fraction": float(np.mean([s.r_size / s.n for s in stats])), "nnz_last": stats[-1].nnz,
        "m2_last": stats[-1].m2, "q_last": stats[-1].q,
        "ms_merge": float(np.mean([s.ms_merge for s in stats])),
        "ms_screen": float(np.mean([s.ms_screen for s in stats])),
        "ms_local_move": float(np.mean([s.ms_local_move for s in stats])),
        "ms_coarsen": float(np.mean([s.ms_coarsen for s in stats])),
        "coarse0_delta_steps": int(sum(s.coarse0_delta for s in stats)),
        "coarse0_entries_mean": float(np.mean([s.coarse0_entries for s in stats])),
        "level0_local_move_gbs": gbs, "level0_frac": (gbs / peak) if gbs else None, "peak_kind": peak_kind,
        "timing": "CUDA events on the context stream around each update", "clocks": clk.summary(),
    }


# ------------------------------------------------------------------ learned screen

def learned_arm(args):
    print(json.dumps(learned_leg(args)), flush=True)


def learned_leg(args):
    """Learned screen vs plain Delta-screening: train the network on move labels
    of full re-evaluation (BASE) runs of the LFR generator at n = 200,000
    (--train-seeds runs of 12 steps), then run each evaluation stream (fresh
    seeds of LFR n = 2,000,000 and of R-MAT scale 24) three times: plain
    Delta-screening, the learned screen, and the learned screen with the judge
    (plain Delta-screening from the same state; a step more than 1e-3 below it
    is redone)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd, synth

    torch.cuda.set_device(0)
    T = LFR_STEPS  # the evaluation streams are the 12-step configurations
    warm = min(args.warmup, LFR_STEPS - 2)
    Xs, ys = [], []
    t0 = time.time()
    for r in range(args.train_seeds):
        n_tr = 200_000
        s = synth.lfr(synth.seed_for(4, r), n_tr, int(31.5 * n_tr), 12, kmax=5000.0, smax=12_500.0)
        ctx = dcd.Context(n_tr, mode=dcd.MODE_BASE)
        ctx.set_collect(True)
        for t, (ins, dels) in enumerate(s.steps):
            ctx.apply_batch(ins, dels)
            ctx.update(labels_out=None)
            if t > 0:
                X, y, _ = ctx.screen_data()
                Xs.append(X)
                ys.append(y)
        ctx.close()
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    perm = np.random.default_rng(0).permutation(len(X))
    dX = torch.from_numpy(X[perm]).cuda()
    dy = torch.from_numpy(y[perm]).cuda()
    mlp = dcd.Mlp(seed=11)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    loss = mlp.train(dX, dy, len(X), batch=8192, epochs=args.epochs, lr=2e-3)
    ev1.record()
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    gen_s = time.time() - t0

    def evaluate(name, stream, desc):
        n = stream.n
        T = len(stream.steps)
        d_ins = [torch.from_numpy(np.ascontiguousarray(i)).cuda() for i, _ in stream.steps]
        d_del = []
        for _, dels in stream.steps:
            dd = np.zeros((len(dels), 3), np.int32)
            dd[:, :2] = dels
            d_del.append(torch.from_numpy(dd).cuda())

        ts = torch.cuda.current_stream()

        def run(mode, judge):
            ctx = dcd.Context(n, mode=mode, stream=ts)
            if mode == dcd.MODE_LEARNED:
                ctx.set_screen(mlp, theta_keep=args.theta_keep, theta_add=args.theta_add, judge=judge)
            out = []
            for t in range(T):
                ctx.apply_batch_device(d_ins[t], len(stream.steps[t][0]), d_del[t], len(stream.steps[t][1]))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ts)
                _, q, st = ctx.update(labels_out=None)
                e1.record(ts)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if t == 0:
                    ctx.autotune(reps=2)
                if t >= 1 + warm:
                    out.append((ms, q, st.r_size, st.r_screen, st.fallback, st.q_screen, st.pool))
            ctx.close()
            return out

        with ClockSampler(0) as clk:
            plain = run(dcd.MODE_DELTA, False)
            learned = run(dcd.MODE_LEARNED, False)
            judged = run(dcd.MODE_LEARNED, True)
        clocks = clk.summary()
        del d_ins, d_del
        gap = [p[1] - l[1] for p, l in zip(plain, learned)]
        return {
            "workload": name, "description": desc, "timed_steps": f"t={2 + warm}..{T}",
            "r_fraction_delta": float(np.mean([p[2] for p in plain]) / n),
            "r_fraction_learned": float(np.mean([l[2] for l in learned]) / n),
            "pool_fraction": float(np.mean([l[6] for l in learned]) / n),
            "ms_per_step_delta": float(np.mean([p[0] for p in plain])),
            "ms_per_step_learned": float(np.mean([l[0] for l in learned])),
            "ms_per_step_learned_judged": float(np.mean([j[0] for j in judged])),
            "q_delta_last": plain[-1][1], "q_learned_last": learned[-1][1],
            "q_gap_max": float(max(gap)), "q_gap_mean": float(np.mean(gap)),
            "steps_within_1e-3": int(sum(g <= 1e-3 for g in gap)), "steps": len(gap),
            "judged_fallbacks": int(sum(j[4] for j in judged)),
            "timing": "CUDA events on the work stream around each update",
            "clocks": clocks,
        }

    evals = []
    for name in args.eval.split(","):
        if name == "lfr":
            st_ = make_stream(args.n, T, replica=9)
            evals.append(evaluate("lfr", st_, workload_desc(st_.n).replace("lfr_2m", f"lfr n={st_.n:,}")))
        elif name == "rmat":
            st_ = synth.rmat(synth.seed_for(2, 9), scale=args.rmat_scale, edge_factor=16, steps=T,
                             ins_frac=0.01, del_frac=0.005)
            evals.append(evaluate("rmat", st_, (f"R-MAT scale {args.rmat_scale} (a=0.57, b=c=0.19), edge factor 16, "
                                                f"weights 1..8, {T} steps of 1% inserts and 0.5% deletes")))
        del st_
    line = {
        "metric": "learned screen vs Delta-screening: |R_t|, ms per step, modularity gap",
        "training": {"runs": args.train_seeds, "n": 200_000, "steps": 12, "rows": int(len(X)),
                     "positive_fraction": float(y.mean()), "epochs": args.epochs, "final_loss": loss,
                     "train_ms_gpu": train_ms, "data_s": gen_s},
        "thresholds": {"keep": args.theta_keep, "add": args.theta_add},
        "evaluations": evals,
    }
    return line


# ------------------------------------------------------------------ batched form

def batched_arm(args):
    line = batched_leg(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def batched_leg(args):
    """512 independent temporal SBMs (n log-uniform in 500..200,000, blocks of
    20..2,000, mean degree 8..32, 3 % inserts and 1 % deletes per step) advanced
    together by one group update per step, against the same graphs updated one
    context at a time (both on the GPU, Delta-screening mode).  Under torchrun
    every rank takes its share of the graphs (no data crosses ranks); the
    job's time per step is the slowest rank's."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1904_08553_gb300 import dcd, shard, synth

    params = synth.batched_params(synth.seed_for(3, 0), args.graphs)
    cost = [int(n * deg) for n, deg, _ in params]
    mine = shard.partition_graphs(cost, world)[rank]
    t0 = time.time()
    streams = synth.batched_sbm(G=args.graphs, steps=7, graphs=set(mine))
    gen_s = time.time() - t0
    sizes = [s.n for s in streams]
    T = len(streams[0].steps)
    ts = torch.cuda.current_stream(dev)

    def timed(fn):
        """CUDA-event time (ms) of fn on the work stream, synchronised on both sides."""
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ts)
        r = fn()
        e1.record(ts)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    grp = dcd.Group(sizes, mode=dcd.MODE_DELTA, stream=ts)
    group_ms = []
    launches_group = []
    with ClockSampler(local) as clk:
        for t in range(T):
            for g, s in enumerate(streams):
                grp.apply_batch(g, *s.steps[t])
            if world > 1:
                dist.barrier()
            l0 = dcd.dcd_kernel_launches()
            ms, (_, q, st) = timed(lambda: grp.update(labels_out=None))
            ms = shard.max_over_ranks(ms, device=dev)
            if t >= 1:
                group_ms.append(ms)
                launches_group.append(dcd.dcd_kernel_launches() - l0)
            else:
                grp.autotune(reps=3)  # degree-bin plan of the union graph (untimed)
    clocks = clk.summary()
    plan = grp.bins()
    q_group = q.copy()
    grp.close()
    # one context per graph, one graph after the other (a context lives for its
    # graph's whole stream); the per-step time is summed over the graphs
    seq_ms = np.zeros(T - 1)
    q_seq = np.zeros(len(sizes))
    launches_seq = 0
    for g, s_ in enumerate(streams):
        ctx = dcd.Context(sizes[g], mode=dcd.MODE_DELTA, stream=ts)
        for t in range(T):
            ctx.apply_batch(*s_.steps[t])
            l0 = dcd.dcd_kernel_launches()
            ms, (_, q_seq[g], stg) = timed(lambda: ctx.update(labels_out=None))
            if t >= 1:
                seq_ms[t - 1] += ms
            if t == T - 1:
                launches_seq += dcd.dcd_kernel_launches() - l0
        ctx.close()
    seq_mean = shard.max_over_ranks(float(np.mean(seq_ms)), device=dev)
    same = shard.sum_over_ranks(float(not np.array_equal(q_group, q_seq)), device=dev) == 0
    n_all = int(shard.sum_over_ranks(float(sum(sizes)), device=dev))
    if world > 1 and not args.keep_pg:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return None
    line = {
        "metric": "batched form: ms per time step for all graphs (group update vs one context per graph)",
        "workload": (f"{args.graphs} temporal SBMs, n log-uniform 500..200,000 (total {n_all:,} vertices), "
                     f"initial load + {T - 1} steps of 3% inserts / 1% deletes"),
        "n_gpus": world, "scaling": "strong" if world > 1 else None,
        "ms_per_step_group": float(np.mean(group_ms)), "ms_per_step_one_at_a_time": seq_mean,
        "speedup": float(seq_mean / np.mean(group_ms)),
        "kernel_launches_per_step": {"group": float(np.mean(launches_group)), "one_at_a_time": int(launches_seq)},
        "timing": "CUDA events on the work stream around each update, synchronised on both sides",
        "clocks": clocks,
        "identical_modularity": bool(same), "generation_s": gen_s,
        "bin_plan": {"variants": plan[0], "max_degree": plan[1]},
    }
    return line


# ------------------------------------------------------------ temporal resolution

RES_FINE_STEPS = 28
RES_BINS = (2, 4, 8, 12, 16, 20, 24, 28)


def resolution_stream(n: int, replica: int = 0):
    """An insert-only LFR-style interaction stream of 28 fine steps (no drift,
    no deletes: the shape of a temporal interaction log), LFR_EVENTS scaled by
    n / LFR_N."""
    from paper_1904_08553_gb300 import synth

    synth.build()
    events = int(round(LFR_EVENTS * n / LFR_N))
    return synth.lfr(synth.seed_for(5, replica), n, events, RES_FINE_STEPS, kmax=min(20_000.0, n / 2),
                     smax=min(50_000.0, n / 4), drift=0.0, del_frac=0.0)


def resolution_sweep(make_ctx, fine, ks, modes):
    """The temporal-resolution experiment of Sec. IV-C on one insert-only
    stream: for every binning k of it and every mode, a fresh context runs the
    k steps.  make_ctx(n, mode) returns an object with step(ins, dels) ->
    (Q, ms, |R_t|) and close().  Rows: k, mode, total ms, mean Q over the
    steps, mean |R_t| / n."""
    from paper_1904_08553_gb300 import synth

    rows = []
    for k in ks:
        s = synth.rebin(fine, k)
        for mode in modes:
            ctx = make_ctx(s.n, mode)
            qs, ms, rs = [], [], []
            for ins, dels in s.steps:
                q, t_ms, r = ctx.step(ins, dels)
                qs.append(q)
                ms.append(t_ms)
                rs.append(r / s.n)
            ctx.close()
            rows.append({"steps": k, "mode": mode, "total_ms": float(sum(ms)), "mean_q": float(np.mean(qs)),
                         "mean_r_fraction": float(np.mean(rs))})
    return rows


def resolution_arm(args):
    """Sweep on the GPU: Delta-screening against dLouvain-base at every
    binning; reports the savings and mean modularity per number of steps."""
    import torch

    from paper_1904_08553_gb300 import dcd

    dcd.lib()
    torch.cuda.set_device(0)
    fine = resolution_stream(args.n)

    class Ctx:
        def __init__(self, n, mode):
            self.c = dcd.Context(n, mode={"base": dcd.MODE_BASE, "delta": dcd.MODE_DELTA}[mode])

        def step(self, ins, dels):
            self.c.apply_batch(ins, dels)
            _, q, st = self.c.update(labels_out=None)
            return q, st.ms_total, st.r_size

        def close(self):
            self.c.close()

    rows = resolution_sweep(Ctx, fine, RES_BINS, ("base", "delta"))
    table = []
    for k in RES_BINS:
        b = next(r for r in rows if r["steps"] == k and r["mode"] == "base")
        d = next(r for r in rows if r["steps"] == k and r["mode"] == "delta")
        table.append({"steps": k, "ms_base": b["total_ms"], "ms_delta": d["total_ms"],
                      "savings_pct": 100.0 * (1.0 - d["total_ms"] / b["total_ms"]) if b["total_ms"] > 0 else None,
                      "mean_q_base": b["mean_q"], "mean_q_delta": d["mean_q"],
                      "mean_r_fraction_delta": d["mean_r_fraction"]})
    print(json.dumps({
        "metric": "temporal-resolution sweep: Delta-screening savings and mean modularity per number of steps",
        "workload": (f"insert-only LFR-style stream, n={args.n:,}, {sum(len(i) for i, _ in fine.steps):,} "
                     f"events in {RES_FINE_STEPS} fine steps, rebinned into k steps"),
        "n_gpus": 1, "unit": "ms (device time of the updates, all steps)", "rows": table,
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="main line only: skip the R-MAT, batched and learned-screen legs")
    ap.add_argument("--keep-pg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default degree-bin plan (a fixed kernel sequence, for profiling)")
    ap.add_argument("--n", type=int, default=LFR_N, help="vertex count (smaller cases for profiling)")
    ap.add_argument("--pass-loop", default="device", choices=["device", "host"],
                    help="host: the host enqueues each local-move pass (dcd_config.pass_loop = 1) instead of "
                         "one graph launch per level, so that a kernel profiler lists the pass kernels too")
    ap.add_argument("--autotune-at", type=int, default=1,
                    help="tune the degree-bin plan after this many steps (at most 1 + warm-up; untimed). "
                         "The tuner evaluates every vertex once per candidate plan outside the pass-loop "
                         "graph, so a later step gives a profiler the local-move kernels on a larger graph")
    ap.add_argument("--workload", default="lfr_2m", choices=["lfr_2m", "learned", "batched", "resolution"])
    ap.add_argument("--graphs", type=int, default=512)
    ap.add_argument("--train-seeds", type=int, default=40)
    ap.add_argument("--eval", default="lfr,rmat", help="learned workload: evaluation streams (lfr, rmat)")
    ap.add_argument("--rmat-scale", type=int, default=24)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--theta-keep", type=float, default=0.3)
    ap.add_argument("--theta-add", type=float, default=0.9)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "lfr_2m" and args.warmup > LFR_STEPS - 2:
        ap.error(f"--warmup must leave a timed step of the {LFR_STEPS}-step configuration (at most {LFR_STEPS - 2})")
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "learned":
        learned_arm(args)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "resolution":
        resolution_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
