#!/usr/bin/env python3
"""Benchmark of the relocalization scoring path on GB300.

One step = one pass of the whole path over the warehouse workload (4096x4096
grid at 0.05 m, 20000 RRT hypotheses, 1440-beam 360-degree noisy scan, 720
orientations, TAM on the SMAD top 1024; --config 1 takes the office
workload instead): EDT map precompute, scan preparation, ray cast + SMAD for
every hypothesis, SMAD top-K, batched TAM over every orientation of every
survivor, orientation argmax, local top-k.

value: hypothesis x orientation evaluations (SMAD + TAM) per second with all
inputs resident in HBM; each step is timed with CUDA events on the library's
stream and L2 is flushed (256 MiB write) before every timed step.
e2e: the same metric through the host entry points (relo_update_map,
relo_set_hypotheses, relo_relocalize) from pinned host buffers, host<->device
copies included, wall-clock per step.
batched / served: the same line also carries the batched form (64 mixed
requests per step in one launch per stage) and the served form (Poisson
arrivals against 8 resident maps: best relocalizations/s at p99 <= 50 ms,
continuous batching against the one-request-at-a-time pipeline, with and
without resident tables).

--impl reference times the FP64 CPU oracle on the host cores, each step a
bounded sample of the same workload (its value is the sample's evaluations
over the sample's measured time, nothing extrapolated).
"""
from __future__ import annotations

import argparse
import faulthandler
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hypothesis×orientation evals/s (SMAD+TAM); relocalizations/s at p99 latency"
UNIT = "evals/s"
ROOFLINE_STAGES = ["raycast", "smad", "tam"]   # kernels timed inside the timed region for their roofline
SIDE_STAGES = ("edt_field",)   # stages the library runs on its side stream
OFFICE = 1      # the office workload (sweep, table2, rrt)
DATA = {1: "synthetic (seeded office map, RRT hypotheses, noisy LiDAR scan)",
        2: "synthetic (seeded warehouse map, RRT hypotheses, noisy LiDAR scan)"}
WORKLOADS = {
    1: ("office 1024x1024 @0.05 m, 5000 RRT hypotheses x 360 orientations, 1081-beam 270-deg noisy scan "
        "(N_s 1440), TAM on SMAD top 256 (all batches scored)"),
    2: ("warehouse 4096x4096 @0.05 m, 20000 RRT hypotheses x 720 orientations, 1440-beam 360-deg noisy scan "
        "(N_s 1440), TAM on SMAD top 1024 (all batches scored)"),
}
# Integer operations of one DDA cell step of the definition (Eq. 13): an
# error-term update, a compare, a step in x or y, an occupancy test and the
# loop test come to about 8-10, and ncu on a cell-by-cell walk of the office
# counted 10.1 thread instructions per step.  The tile walk crosses empty
# tiles and boxes of tiles without visiting their cells, so this measures the
# definition's work, which the kernel does with fewer instructions; the ray
# cast's roofline itself counts the instructions it executes (ncu, per launch).
OPS_PER_DDA_STEP = 10
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=sorted(WORKLOADS),
                    help="single-request workload: 2 = warehouse 4096^2 (default), 1 = office 1024^2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="e2e steps (default: min(steps, 200))")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "served", "sweep", "rrt", "table2", "table3"],
                    help="single: one request per step on --config's workload (default; the line also carries the "
                         "batched and served forms unless --no-extras); batched: 64 mixed requests per step; "
                         "served: Poisson arrivals against 8 resident maps")
    ap.add_argument("--no-extras", action="store_true", help="single: leave out the batched and served forms")
    ap.add_argument("--tune", action="store_true",
                    help="batched / single: run the launch-shape autotuner first and update its cache for this GPU")
    ap.add_argument("--extra-steps", type=int, default=10, help="single: timed steps of the batched form")
    ap.add_argument("--rates", default="",
                    help="served: arrival rates per second (default: a ladder that grows by 1.5x from 250/s until "
                         "p99 passes 50 ms, then bisects the last step twice)")
    ap.add_argument("--duration", type=float, default=2.0, help="served: seconds of arrivals per rate")
    ap.add_argument("--coarse", default="smad", choices=["smad", "caer", "smad_direct"],
                    help="single workload: ranking metric, SMAD (Eq. 19-20), CAER (Eq. 21) or SMAD by direct "
                         "window sums (the Table II ablation without prefix sums); the rooflines assume SMAD")
    ap.add_argument("--fine", default="tam", choices=["tam", "tam_mean", "baseline", "lf"],
                    help="single workload: scoring metric, TAM (Eq. 31), TAM_mean (Eq. 34), wp_baseline (Eq. 33) "
                         "or wp_LF (Eq. 32)")
    ap.add_argument("--icp-iters", type=int, default=0,
                    help="single workload: ICP iterations per local top-k pose before its re-evaluation (0: none)")
    ap.add_argument("--serve-configs", default="16x3",
                    help="served: max_batch x max_inflight settings to measure (the best is reported)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world):
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo")
        return dist
    return None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# our GPU path
# ---------------------------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def committed_traffic(stage: str, config: int, key: str = "dram_bytes_per_launch"):
    """DRAM (or, with key, L2) bytes per launch from the committed ncu summary
    of this workload, if the kernel source is unchanged since the capture
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(f"config{config}", {}).get(stage)
    except (OSError, ValueError, AttributeError):
        return None
    if not rec:
        return None
    try:
        h = code_sha(os.path.join(ROOT, "paper_2511_01219_gb300", "csrc", rec["source"]))
    except OSError:
        return None
    return rec.get(key) if h == rec["code_sha"] else None


def code_sha(path: str) -> str:
    """sha256[:16] of a CUDA source with its comments and whitespace removed, so
    that a counter capture stays matched to the code it measured through edits
    of the comments only."""
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()[:16]


def apply_tuning(ctx, torch, local) -> dict:
    """Loads the autotuner's cached launch shapes for this GPU into ctx, if a
    cache exists (paper_2511_01219_gb300/tuning/<device>.json)."""
    from paper_2511_01219_gb300 import autotune
    path = autotune.cache_path(torch.cuda.get_device_name(local))
    entries = autotune.load(path)
    if entries:
        ctx.set_tuning(entries)
    return {"source": os.path.relpath(path, ROOT) if entries else None, "entries": len(entries)}


def run_ours(args, world, rank, local, dist):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(args.config)
    # a high-priority stream for the request path, so the map update's field pass (on the library's low-priority
    # side stream) yields to the ray cast and SMAD
    stream = torch.cuda.Stream(priority=-1)
    torch.cuda.set_stream(stream)
    ctx = relo.Relo(n_orient=wl.n_orient, topk=wl.topk, early_stop=0, stream=stream,
                    coarse_metric=["smad", "caer", "smad_direct"].index(args.coarse),
                    fine_metric=["tam", "tam_mean", "baseline", "lf"].index(args.fine), icp_iters=args.icp_iters)
    grid_d = torch.tensor(wl.grid, device="cuda")
    hyps_d = torch.tensor(wl.hyps, device="cuda")
    z_d = torch.tensor(wl.ranges, device="cuda")
    res_d = torch.empty(relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    mid = ctx.load_map_dev(grid_d, wl.res)
    ctx.set_hypotheses_cells_dev(mid, hyps_d)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    tuning = apply_tuning(ctx, torch, local)

    def step():
        ctx.update_map_dev(mid, grid_d)
        ctx.relocalize_dev(mid, z_d, wl.angles, wl.max_range, res_d)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if args.tune:
        from paper_2511_01219_gb300 import autotune
        cache = autotune.cache_path(torch.cuda.get_device_name(local))
        res_tune = autotune.tune(ctx, step, [(len(wl.ranges), wl.n_orient, min(wl.topk, len(wl.hyps)))],
                                 log=lambda s: print(s, file=sys.stderr), single=True)
        merged = {(k, tuple(key)): val for k, key, val in autotune.load(cache)}
        merged.update({(k, tuple(key)): val for k, key, val in res_tune["entries"]})
        autotune.save(cache, [(k, key, val) for (k, key), val in merged.items()],
                      {"device": torch.cuda.get_device_name(local), "workloads": "batched + single"})
        tuning = apply_tuning(ctx, torch, local)
        tuning["tuning_run"] = {"tam_ms": res_tune["tam_ms"], "cast_ms": res_tune["cast_ms"],
                                "seconds": res_tune["seconds"], "trials": len(res_tune["trials"])}
        for _ in range(2):
            step()
        torch.cuda.synchronize()
    r = relo.result_from_bytes(bytes(res_d.cpu().numpy()))
    if r.status != relo.OK:
        raise RuntimeError(f"relocalization failed with status {r.status}")
    evals_per_step = int(r.n_smad_evals + r.n_tam_evals)

    # Inside the timed region only the kernels with a roofline are bracketed by
    # events (each event pair costs the stream time); the other stages' times
    # come from a separate pass below.
    ctx.set_profiling_stages(ROOFLINE_STAGES)
    ctx.stage_times(reset=True)
    k0 = ctx.kernels_launched()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(dist)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(dist)
    per_step = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(per_step)
    stage_ms, stage_n, k1 = ctx.stage_times(reset=True)
    launches = k1 - k0
    t_max = max_over_ranks(dist, total_ms)
    evals_all = sum_over_ranks(dist, float(evals_per_step * args.steps))
    value = evals_all / (t_max / 1e3)
    # every stage bracketed, untimed: the per-stage breakdown
    n_bd = min(args.steps, 50)
    ctx.set_profiling(True)
    for i in range(n_bd):
        flush.fill_(i & 0xFF)
        step()
    bd_ms, _, _ = ctx.stage_times(reset=True)
    ctx.set_profiling(False)

    # dominant kernel and its roofline
    info = ctx.scan_info()
    n_valid, n_orient, K = info[3], info[1], info[6]
    peaks, peak_kind = measured_peaks()
    l2 = relo.probe_l2()
    # the EDT's field pass runs on the library's side stream beside the ray cast: its event time is
    # wall time on shared SMs, so the shares and the dominant kernel are over the main stream's stages
    main_ms = {k: v for k, v in bd_ms.items() if k not in SIDE_STAGES}
    bd_total = sum(main_ms.values())
    shares = {k: v / bd_total for k, v in main_ms.items()}
    dominant = max(main_ms, key=main_ms.get)
    tam_bytes = 2.0 * n_valid * K * n_orient * args.steps          # 2 B field read per valid beam per (h, m)
    hbm = peaks["hbm_gbs"]
    roof = {}
    if stage_ms["tam"] > 0:
        gbs = tam_bytes / (stage_ms["tam"] / 1e3) / 1e9
        roof["tam"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(gbs / hbm, 4),
                       # the counters were taken with TAM scoring; the other metrics run another epilogue
                       "traffic": committed_traffic("tam", args.config) if args.fine == "tam" else None,
                       "peak_source": f"{peak_kind} hbm_gbs",
                       "frac_hbm": round(gbs / hbm, 4),
                       "gathers_per_s": round(gbs * 1e9 / 2.0),
                       # the gathers against the rate of 2-byte gathers with no locality at all
                       "frac_random_gather": round(gbs / l2["gather_2b_gbs"], 4),
                       "random_gather_peak_per_s": round(l2["gather_per_s"]),
                       "avg_launch_ms": round(stage_ms["tam"] / max(stage_n["tam"], 1), 4)}
        # the L2 -> SM bytes the kernel really moves (ncu, per launch) against the streaming L2 rate
        l2b = committed_traffic("tam", args.config, key="l2_bytes_per_launch") if args.fine == "tam" else None
        roof["tam"]["l2_traffic"] = l2b
        roof["tam"]["frac_l2"] = (round(l2b / (roof["tam"]["avg_launch_ms"] / 1e3) / 1e9 / l2["stream_gbs"], 4)
                                  if l2b else None)
        roof["tam"]["l2_peak"] = round(l2["stream_gbs"], 1)
        roof["tam"]["l2_peak_source"] = "streaming 16-byte reads of an L2-resident buffer (relo_probe_l2_stream)"
        # what bounds the gathers: the L1 data path's busy share in the committed ncu capture of this kernel
        l1 = committed_traffic("tam", args.config, key="l1_busy_pct") if args.fine == "tam" else None
        roof["tam"]["l1_data_path_busy"] = round(l1 / 100.0, 4) if l1 else None
        roof["tam"]["l1_source"] = "ncu l1tex__throughput.avg.pct_of_peak_sustained_active, profiles/traffic.json"
    dda = info[8]
    if stage_ms["raycast"] > 0 and dda:
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        peak_tops = 128 * sm_count * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        avg_ms = stage_ms["raycast"] / max(stage_n["raycast"], 1)
        dda_tops = dda * OPS_PER_DDA_STEP * args.steps / (stage_ms["raycast"] / 1e3) / 1e12
        # thread instructions one launch executes (ncu), if the kernel is unchanged since the capture
        inst = committed_traffic("raycast", args.config, key="thread_inst_per_launch") if args.coarse == "smad" else None
        tops = inst / (avg_ms / 1e3) / 1e12 if inst else dda_tops
        roof["raycast"] = {"bound": "alu", "achieved": round(tops, 3), "peak": round(peak_tops, 2),
                           "unit": "Tops/s", "frac": round(tops / peak_tops, 4),
                           "basis": ("executed thread instructions per launch (ncu) / live launch time" if inst else
                                     f"{OPS_PER_DDA_STEP} integer operations per DDA cell step of the definition "
                                     "(no current instruction count)"),
                           "thread_inst_per_launch": inst,
                           "traffic": committed_traffic("raycast", args.config),
                           "peak_source": f"128 int32 lanes x {sm_count} SMs x {peaks.get('sm_max_mhz')} MHz",
                           # the definition's work: above 1 when whole tiles and boxes are crossed in one move
                           "dda_ops_per_s": round(dda_tops * 1e12),
                           "frac_dda": round(dda_tops / peak_tops, 4),
                           "ops_per_dda_step": OPS_PER_DDA_STEP,
                           "dda_steps_per_step": dda,
                           "avg_launch_ms": round(avg_ms, 4)}
    if stage_ms["smad"] > 0:
        smad_bytes = 4.0 * info[0] * info[9] * args.steps          # one Q16 range per (hypothesis, direction)
        gbs = smad_bytes / (stage_ms["smad"] / 1e3) / 1e9
        roof["smad"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(gbs / hbm, 4),
                        # the counters are the prefix-sum SMAD kernel's; other rankings run other code
                        "traffic": committed_traffic("smad", args.config) if args.coarse == "smad" else None,
                        "peak_source": f"{peak_kind} hbm_gbs",
                        "frac_hbm": round(gbs / hbm, 4),
                        "frac_l2": round(gbs / l2["stream_gbs"], 4),
                        "l2_peak": round(l2["stream_gbs"], 1),
                        "l2_peak_source": "streaming 16-byte reads of an L2-resident buffer (relo_probe_l2_stream)",
                        "avg_launch_ms": round(stage_ms["smad"] / max(stage_n["smad"], 1), 4)}
    main_roof = roof.get(dominant) or roof.get("tam")
    pct = sorted(per_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": DATA[args.config],
        "config": {"workload": WORKLOADS[args.config], "map": list(wl.grid.shape), "n_hyp": len(wl.hyps),
                   "n_orient": wl.n_orient, "n_beams": len(wl.ranges), "n_s": wl.n_s, "topk": wl.topk,
                   "evals_per_step": evals_per_step, "l2": "flushed before every timed step (256 MiB write)",
                   "timed_step": "map update from a device grid and its EDT, scan preparation, ray cast, SMAD, "
                                 "top-K, TAM, selection (hypotheses stay resident; e2e uploads map, hypotheses and "
                                 "scan from host buffers every step); the ray direction tables (k_ray_tables, once "
                                 "per sensor geometry) are built before the timed region",
                   "ranking": args.coarse, "scoring": args.fine, "icp_iters": args.icp_iters,
                   "parallelism": f"replicas x{world}"},
        "relocalizations_per_s": world * args.steps / (t_max / 1e3),
        "latency_ms": {"p50": pct[len(pct) // 2], "p99": pct[min(len(pct) - 1, int(math.ceil(0.99 * len(pct))) - 1)]},
        "gpu_launches": int(launches),
        "stage_ms_per_step": {k: round(v / n_bd, 5) for k, v in bd_ms.items()},
        "stage_share": {k: round(v, 4) for k, v in shares.items()},
        "stage_times": f"stage_ms_per_step and stage_share from {n_bd} further steps with every kernel bracketed by "
                       f"events; the timed steps bracket only {', '.join(ROOFLINE_STAGES)} (the roofline kernels); "
                       f"{', '.join(SIDE_STAGES)} runs on the side stream beside the ray cast and is left out of the "
                       f"shares",
        "dominant_kernel": dominant,
        "roofline": main_roof,
        "roofline_all": roof,
        "clocks": clk,
        "tuning": tuning,
    }
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, ctx, mid, wl, relo, torch, flush, dist, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    line["l2_probe"] = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in l2.items()}
    ctx.close()
    del flush
    if not args.no_extras:
        b = run_batched(args, world, rank, local, dist, steps=args.extra_steps)
        line["batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "relocalizations_per_s", "latency_ms",
                                             "gpu_launches", "stage_ms_per_step", "clocks", "launch_shapes",
                                             "resident_tables")}
        line["batched"]["workload"] = b["config"]["workload"]
        line["batched"]["steps"] = b["steps"]
        line["batched"]["evals_per_step"] = b["config"]["evals_per_step"]
        sv = run_served(args, world, rank, local, dist)
        line["served"] = {k: sv[k] for k in ("value", "unit", "best_rate_p99_le_50ms", "seconds_per_rate",
                                             "pose_agreement", "pool")}
        line["served"]["workload"] = sv["config"]["workload"]
        line["served"]["ladders"] = {m: sv[m] for m in sv["modes"]}
    return line


def run_e2e(args, ctx, mid, wl, relo, torch, flush, dist, world):
    """Same metric through the host API with pinned inputs copied every step."""
    import numpy as np
    n_steps = args.e2e_steps or min(args.steps, 200)
    grid_h = torch.from_numpy(np.ascontiguousarray(wl.grid)).pin_memory()
    xy_h = torch.from_numpy(np.ascontiguousarray(
        (wl.hyps.astype(np.float64) + 0.5) * wl.res)).pin_memory()
    z_h = torch.from_numpy(np.ascontiguousarray(wl.ranges)).pin_memory()
    out = relo.Result()

    def step():
        ctx.update_map_ptr(mid, grid_h.data_ptr())
        ctx.set_hypotheses_ptr(mid, xy_h.data_ptr(), len(wl.hyps))
        ctx.relocalize_ptr(mid, z_h.data_ptr(), wl.angles, len(wl.ranges), wl.max_range, out)

    for _ in range(3):
        step()
    evals = int(out.n_smad_evals + out.n_tam_evals)
    barrier(dist)
    total = 0.0
    for i in range(n_steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        total += time.perf_counter() - t0
    barrier(dist)
    t_max = max_over_ranks(dist, total)
    e = sum_over_ranks(dist, float(evals * n_steps)) / t_max
    h2d = wl.grid.size + 8 * len(wl.hyps) + 4 * len(wl.ranges)
    d2h = relo.RESULT_BYTES + 4
    return {"value": e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": n_steps, "ms_per_step": 1e3 * t_max / n_steps, "timing": "wall clock per blocking step"}


# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------------------

def oracle_step(wl, n_smad: int, n_tam_hyp: int, threads: int):
    """One pass of the oracle over a sample of the workload: the EDT of the
    whole map, SMAD of n_smad hypotheses spread over the set, and TAM of
    n_tam_hyp hypotheses (standing in for as many survivors: the cost does not
    depend on which) x every orientation.  Returns (evaluations made, seconds,
    description); nothing is scaled."""
    import numpy as np

    import oracle
    prm = oracle.Params(n_orient=wl.n_orient, topk=wl.topk)
    t0 = time.perf_counter()
    d2 = oracle.edt(wl.grid, threads)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    sel = np.arange(0, len(wl.hyps), max(1, len(wl.hyps) // n_smad))[:n_smad]
    oracle.smad(wl.grid, wl.hyps[sel], pl, threads)
    oracle.tam_grid(wl.grid, wl.hyps, np.arange(n_tam_hyp), pl, prm, wl.res, d2, threads)
    dt = time.perf_counter() - t0
    n_m = 1 if pl["panoramic"] else pl["n_orient"]
    evals = len(sel) * n_m + n_tam_hyp * pl["n_orient"]
    full = len(sel) == len(wl.hyps) and n_tam_hyp == min(wl.topk, len(wl.hyps))
    desc = (f"{'the full step' if full else 'a sample of the step'}: EDT of the whole map + SMAD of "
            f"{len(sel)}/{len(wl.hyps)} hypotheses + TAM of {n_tam_hyp} hypotheses x {pl['n_orient']} orientations "
            f"({'as many as the survivors' if full else 'the step scores ' + str(min(wl.topk, len(wl.hyps)))}); "
            "value = evaluations made / measured time, no scaling")
    return evals, dt, desc


def cpu_baseline(wl, repeats: int = 3):
    """The oracle on all host cores over the whole step (every hypothesis's
    SMAD, TAM of as many hypotheses as the step has survivors), the median of
    a few passes (about 3 s each on the warehouse)."""
    import oracle
    threads = oracle.max_threads()
    runs = [oracle_step(wl, n_smad=len(wl.hyps), n_tam_hyp=min(wl.topk, len(wl.hyps)), threads=threads)
            for _ in range(repeats)]
    evals, desc = runs[0][0], runs[0][2]
    dts = [r[1] for r in runs]
    dt = statistics.median(dts)
    return {"value": evals / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc, "s_per_step": dt,
            "passes": repeats, "s_per_pass": [round(x, 4) for x in dts]}


# the reference arm's step: a bounded sample of the workload (about 1-3 s on 16 host cores)
REF_SAMPLE = {1: (1000, 32), 2: (4000, 96)}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import oracle
    import workloads
    oracle.build()
    wl = workloads.config(args.config)
    threads = oracle.max_threads()
    n_smad, n_tam = REF_SAMPLE[args.config]
    for _ in range(max(args.warmup, 0)):
        oracle_step(wl, n_smad, n_tam, threads)
    total_evals, total_s, desc = 0, 0.0, ""
    for _ in range(args.steps):
        e, dt, desc = oracle_step(wl, n_smad, n_tam, threads)
        total_evals += e
        total_s += dt
    value = total_evals / total_s
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": DATA[args.config],
        "config": {"workload": WORKLOADS[args.config], "map": list(wl.grid.shape), "n_hyp": len(wl.hyps),
                   "n_orient": wl.n_orient, "n_beams": len(wl.ranges), "n_s": wl.n_s, "topk": wl.topk,
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_sweep(args, world, rank, local, dist):
    """Translation-affinity sweep in the manner of Fig. 8, on the office map:
    15 positions 0.1 m apart through the scan's true position (along the axis
    whose cells are all free) x 36 orientations 10 degrees apart from the true
    one = 540 poses, scored by each scoring metric (TAM, TAM_mean, wp_baseline,
    wp_LF).  For every position it reports whether the true orientation still
    scores best among the 36, and the time of one sweep."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(OFFICE)
    gx, gy, gth = wl.gt_pose
    cells, offs, axis, sweep_q = workloads.sweep_poses(wl)
    metrics = ["tam", "tam_mean", "baseline", "lf"]
    out = {}
    for fine, name in enumerate(metrics):
        ctx = relo.Relo(n_orient=360, topk=len(cells), batch=len(cells), local_topk=1, early_stop=0, fine_metric=fine)
        mid = ctx.load_map(wl.grid, wl.res)
        ctx.set_hypotheses(mid, workloads.cell_centres(cells.astype(np.int32), wl.res))
        for _ in range(3):
            ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 20
        for _ in range(reps):
            ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
        ms = (time.perf_counter() - t0) * 1e3 / reps
        surv = ctx.stage(relo.STAGE_SURVIVORS, torch.empty(len(cells), dtype=torch.int32, device="cuda")).cpu().numpy()
        T = ctx.stage(relo.STAGE_TAM, torch.empty(len(cells) * 360, dtype=torch.float32, device="cuda"))
        T = T.cpu().numpy().reshape(len(cells), 360)
        rows = np.empty_like(T)
        rows[surv] = T                     # back to position order
        sw = rows[:, sweep_q]              # 15 positions x 36 orientations
        wins = [bool(np.argmax(sw[i]) == 0) for i in range(len(cells))]
        best = np.unravel_index(np.argmax(sw), sw.shape)
        out[name] = {"true_orientation_best_at_offsets_m": [round(float(o) * wl.res, 2) for o, w in zip(offs, wins) if w],
                     "fraction": round(sum(wins) / len(wins), 3),
                     "global_best": {"offset_m": round(float(offs[best[0]]) * wl.res, 2), "orientation_deg": 10 * int(best[1])},
                     "ms_per_sweep": round(ms, 3)}
        ctx.close()
    return {"metric": "translation affinity (true orientation best among 36 at each of 15 offsets)", "value": None,
            "unit": None, "n_gpus": world, "data": "synthetic office map (1024x1024 at 0.05 m) and noisy scan",
            "config": {"workload": f"sweep: 15 positions 0.1 m apart along {axis} x 36 orientations 10 deg apart = 540 poses",
                       "true_pose": [round(float(gx), 3), round(float(gy), 3), round(float(gth), 4)]},
            "metrics": out}


def run_table2(args, world, rank, local, dist):
    """Table II in kind on the office map: the batched loop of Sec. III
    (batches of 200 survivors, local top-20, stop once a batch's best score is
    >= tau = 0.95) over K = min(N_h, 4096) survivors (the largest top-K the
    library takes), with three rankings: SMAD
    with the prefix sums of Eq. 17, SMAD with direct window sums, and none
    (the hypotheses in their own order).  Each of 8 seeded true poses is a
    hypothesis cell and an orientation of the grid; its scan is that cell's
    synthesized scan (the library's ray cast, Eq. 13) read at the beams'
    directions, so the true pose is where the method's own ranges fit
    exactly.  Per arm: mean time per relocalization, batches and TAM
    evaluations run, and how often the true pose was selected."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(OFFICE)
    rng = np.random.default_rng(2511)
    n_enum = wl.n_s // wl.n_orient
    K = min(len(wl.hyps), 4096)
    trials = [(int(rng.integers(len(wl.hyps))), n_enum * int(rng.integers(wl.n_orient))) for _ in range(8)]
    trials = [t for t in trials if t[0] < K]   # every arm must be able to reach the true hypothesis
    b = np.rint(wl.angles.astype(np.float64) / (2.0 * math.pi / wl.n_s)).astype(np.int64) % wl.n_s
    ctx = relo.Relo(n_orient=wl.n_orient)
    mid = ctx.load_map(wl.grid, wl.res)
    cells = torch.tensor(np.array([wl.hyps[h] for h, _ in trials], np.int32), device="cuda")
    rows, _ = ctx.synth_scans(mid, cells, wl.angles, wl.max_range, wl.n_s, with_hits=False)
    rows = rows.cpu().numpy().astype(np.int64)
    ctx.close()
    scans = []
    for t, (h, m) in enumerate(trials):
        q = rows[t, (b + m) % wl.n_s]
        scans.append(np.where(q > 0, q / 65536.0 * wl.res, wl.max_range).astype(np.float32))
    arms = {}
    for name, code in (("smad_prefix_sums", relo.COARSE_SMAD), ("smad_direct_sums", relo.COARSE_SMAD_DIRECT),
                       ("no_ordering", relo.COARSE_NONE)):
        ctx = relo.Relo(n_orient=wl.n_orient, topk=K, batch=200, local_topk=20, tau=0.95, early_stop=1,
                        coarse_metric=code)
        mid = ctx.load_map(wl.grid, wl.res)
        ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
        ms, batches, tam_evals, found = [], [], [], 0
        for (h, m), z in zip(trials, scans):
            for _ in range(3):
                got = ctx.relocalize(mid, z, wl.angles, wl.max_range)
            torch.cuda.synchronize()
            reps = 10
            t0 = time.perf_counter()
            for _ in range(reps):
                got = ctx.relocalize(mid, z, wl.angles, wl.max_range)
            ms.append((time.perf_counter() - t0) * 1e3 / reps)
            batches.append(got.n_batches)
            tam_evals.append(int(got.n_tam_evals))
            found += int(got.hyp == h and got.m == m)
        arms[name] = {"ms_per_relocalization_mean": round(float(np.mean(ms)), 3),
                      "ms_per_relocalization": [round(v, 3) for v in ms], "batches": batches,
                      "tam_evals_mean": round(float(np.mean(tam_evals))), "true_pose_selected": f"{found}/{len(trials)}"}
        ctx.close()
    return {"metric": "Table II in kind: time per relocalization by coarse ranking", "value": None, "unit": None,
            "n_gpus": world, "data": "synthetic office map (1024x1024 at 0.05 m), synthesized scans of 8 seeded poses",
            "config": {"workload": f"table2: {len(wl.hyps)} hypotheses x {wl.n_orient} orientations, K = {K}, "
                                   "batches of 200, local top-20, tau 0.95, early termination",
                       "true_poses": [{"hyp": h, "m": m} for h, m in trials]},
            "arms": arms}


def run_table3(args, world, rank, local, dist):
    """Table III in kind on the office map: the batched loop of Sec. III
    (batches of 200 survivors of the SMAD top-K, local top-20 refined by ICP
    and scored again, early termination at tau = 0.95) with three scoring
    metrics (wp_baseline of
    Eq. 33, TAM_mean of Eq. 34, TAM of Eq. 31) over hypotheses from Algorithm 1
    at rho = 1.0 m and 0.5 m (relo_rrt_sample, from the grid).  Eight seeded
    trial poses on traversable cells with random headings, each with a noisy
    1081-beam 270-degree scan (the office noise model).  Success as in Sec.
    IV-C: position error < 0.5 m and heading error < 30 degrees.  Per arm:
    success rate, mean / std of the time per relocalization (10 repeats per
    trial), batches run."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(OFFICE)
    res, r_robot = wl.res, 0.21
    rng = np.random.default_rng(2513)
    trials = []
    hyp_sets = {}
    clr = workloads.clearance_table(wl.grid, res)
    ok = np.argwhere(clr >= 2 * r_robot)
    p0 = workloads.free_start(wl.grid, res, r_robot, 31, clr)
    ctx0 = relo.Relo()
    for rho in (1.0, 0.5):
        xy, rounds, nodes = ctx0.rrt_sample(wl.grid, res, p0, rho, 0.6, r_robot, 2, seed=31)
        cells = np.unique(np.floor(xy / res).astype(np.int32), axis=0)
        hyp_sets[rho] = cells
    ctx0.close()
    angles = wl.angles
    for t in range(8):
        cy, cx = ok[int(rng.integers(len(ok)))]
        x, y = (cx + rng.uniform(0.1, 0.9)) * res, (cy + rng.uniform(0.1, 0.9)) * res
        th = float(rng.uniform(-math.pi, math.pi))
        z = workloads.add_noise(workloads.render_scan(wl.grid, res, (x, y, th), angles, wl.max_range), wl.max_range,
                                4000 + t)
        trials.append(((x, y, th), z))
    arms = {}
    icp = args.icp_iters if args.icp_iters > 0 else 10   # the local top-k refined as in Sec. III
    for rho, cells in hyp_sets.items():
        K = min(len(cells), 4096)
        for name, code in (("wp_baseline", relo.FINE_BASELINE), ("tam_mean", relo.FINE_TAM_MEAN), ("tam", relo.FINE_TAM)):
            ctx = relo.Relo(n_orient=wl.n_orient, topk=K, batch=200, local_topk=20, tau=0.95, early_stop=1,
                            fine_metric=code, icp_iters=icp)
            mid = ctx.load_map(wl.grid, res)
            ctx.set_hypotheses(mid, workloads.cell_centres(cells, res))
            ms, batches, succ = [], [], 0
            for (x, y, th), z in trials:
                for _ in range(2):
                    got = ctx.relocalize(mid, z, angles, wl.max_range)
                torch.cuda.synchronize()
                reps = 10
                t0 = time.perf_counter()
                for _ in range(reps):
                    got = ctx.relocalize(mid, z, angles, wl.max_range)
                ms.append((time.perf_counter() - t0) * 1e3 / reps)
                batches.append(got.n_batches)
                d_err = math.hypot(got.x - x, got.y - y)
                a_err = abs(math.degrees(math.remainder(got.theta - th, 2 * math.pi)))
                succ += int(d_err < 0.5 and a_err < 30.0)
            arms[f"rho{rho}_{name}"] = {"hypotheses": int(len(cells)), "K": K,
                                        "success_rate": round(succ / len(trials), 3),
                                        "ms_per_relocalization_mean": round(float(np.mean(ms)), 3),
                                        "ms_per_relocalization_std": round(float(np.std(ms)), 3),
                                        "batches": batches}
            ctx.close()
    return {"metric": "Table III in kind: success and time per relocalization by scoring metric and rho",
            "value": None, "unit": None, "n_gpus": world,
            "data": "synthetic office map (1024x1024 at 0.05 m), 8 seeded trial poses with noisy scans",
            "config": {"workload": "table3: RRT hypotheses (relo_rrt_sample) at rho 1.0 and 0.5 m, 360 orientations, "
                                   "batches of 200 of the top K = min(N_h, 4096), local top-20 refined by "
                                   f"{icp} ICP iterations, tau 0.95, early termination; success = position error "
                                   "< 0.5 m and heading error < 30 deg"},
            "arms": arms}


def run_rrt(args, world, rank, local, dist):
    """Hypothesis generation (Algorithm 1) on the office map (1024^2 at 0.05 m,
    rho for about 5000 hypotheses): the GPU sampler (sub-batched nearest-node
    search, in-order resolve: the serial tree for its random points) against
    the serial generator on one host core, with counts, rounds, tree sizes and
    the coverage of the reachable traversable cells."""
    import numpy as np
    import torch
    from scipy.ndimage import label
    from scipy.spatial import cKDTree

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(OFFICE)
    res, r_robot, seed = wl.res, 0.21, 7
    clr = workloads.clearance_table(wl.grid, res)
    p0 = workloads.free_start(wl.grid, res, r_robot, seed, clr)
    rho = math.sqrt(float((clr >= r_robot).sum()) * res * res / (1.1 * 5000))
    lab, _ = label(clr >= r_robot)
    reach = lab == lab[int(p0[1] / res), int(p0[0] / res)]
    ys, xs = np.nonzero(reach)
    cells = np.stack([(xs + 0.5) * res, (ys + 0.5) * res], 1)

    def cover(xy):
        d, _ = cKDTree(np.asarray(xy, np.float64)).query(cells)
        return round(float((d <= rho * math.sqrt(2.0)).mean()), 4)

    t0 = time.perf_counter()
    xs_, n_serial, r_serial = workloads.rrt(wl.grid, res, p0, rho, 0.6, r_robot, 2, seed, clr=clr)
    t_serial = time.perf_counter() - t0
    ctx = relo.Relo()
    clr_d = torch.tensor(clr, device="cuda")
    ctx.rrt_hypotheses(clr_d, res, p0, rho, 0.6, r_robot, 2, seed=seed)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xy, r_gpu, n_gpu = ctx.rrt_hypotheses(clr_d, res, p0, rho, 0.6, r_robot, 2, seed=seed)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    ctx.close()
    return {"metric": "hypothesis generation time (Algorithm 1)", "value": round(t_gpu * 1e3, 2), "unit": "ms",
            "higher_is_better": False, "n_gpus": world, "data": "synthetic office map (1024x1024 at 0.05 m)",
            "config": {"workload": f"rrt: office 1024x1024 @0.05 m, rho {rho:.3f} m, eta_max 0.6 m, r_robot 0.21 m, "
                                   "eps_gain 2"},
            "gpu": {"ms": round(t_gpu * 1e3, 2), "hypotheses": int(len(xy)), "rounds": r_gpu, "nodes": n_gpu,
                    "coverage": cover(xy.cpu().numpy())},
            "serial_cpu": {"ms": round(t_serial * 1e3, 2), "hypotheses": int(len(xs_)), "rounds": r_serial,
                           "nodes": n_serial, "coverage": cover(xs_), "cores": 1}}


def run_batched(args, world, rank, local, dist, steps=None):
    """64 independent relocalizations per step (mixed map sizes, beam counts,
    FoVs and hypothesis counts), one launch per stage, all inputs resident."""
    n_steps = steps or args.steps
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    ins = workloads.batched_instances()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = relo.Relo(n_orient=360, topk=1024, batch=1024, local_topk=20, early_stop=0, stream=stream)
    items = []
    keep = []
    for it in ins:
        g = torch.tensor(it.grid, device="cuda")
        mid = ctx.load_map_dev(g, it.res)
        h = torch.tensor(it.hyps, device="cuda")
        ctx.set_hypotheses_cells_dev(mid, h)
        z = torch.tensor(it.ranges, device="cuda")
        keep += [g, h, z]
        items.append((mid, z, it.angles, it.max_range, it.topk))
    res_t = torch.empty(len(items) * relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    from paper_2511_01219_gb300 import autotune
    cache = autotune.cache_path(torch.cuda.get_device_name(local))

    def one():
        ctx.relocalize_batch_dev(items, res_t)
    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    # the same step with the library's built-in launch shapes, timed alone, before the tuned ones
    builtin_ms = []
    ctx.set_tuning([])
    for i in range(n_steps):
        flush.fill_(i & 0xFF)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        one()
        b_.record(stream)
        b_.synchronize()
        builtin_ms.append(a.elapsed_time(b_))
    shapes = [(len(it.ranges), 360, min(it.topk, len(it.hyps))) for it in ins]
    tuned_info = None
    if getattr(args, "tune", False):
        res_tune = autotune.tune(ctx, one, shapes, log=lambda s: print(s, file=sys.stderr))
        merged = {(k, tuple(key)): val for k, key, val in autotune.load(cache)}
        merged.update({(k, tuple(key)): val for k, key, val in res_tune["entries"]})
        autotune.save(cache, [(k, key, val) for (k, key), val in merged.items()],
                      {"device": torch.cuda.get_device_name(local), "workloads": "batched + single"})
        tuned_info = {"tam_ms": res_tune["tam_ms"], "cast_ms": res_tune["cast_ms"], "seconds": res_tune["seconds"],
                      "trials": len(res_tune["trials"])}
    entries = autotune.load(cache)
    ctx.set_tuning(entries)
    for _ in range(2):
        one()
    torch.cuda.synchronize()
    raw = bytes(res_t.cpu().numpy())
    results = [relo.result_from_bytes(raw[i * relo.RESULT_BYTES:(i + 1) * relo.RESULT_BYTES]) for i in range(len(items))]
    assert all(r.status == relo.OK for r in results), [r.status for r in results]
    evals = sum(int(r.n_smad_evals + r.n_tam_evals) for r in results)
    ctx.set_profiling(True)
    ctx.stage_times(reset=True)
    k0 = ctx.kernels_launched()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
    barrier(dist)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for i in range(n_steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        ctx.relocalize_batch_dev(items, res_t)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(dist)
    per = [a.elapsed_time(b) for a, b in ev]
    total = sum(per)
    stage_ms, stage_n, k1 = ctx.stage_times(reset=True)
    t_max = max_over_ranks(dist, total)
    value = sum_over_ranks(dist, float(evals * n_steps)) / (t_max / 1e3)
    pct = sorted(per)
    ctx.close()
    # The same requests against resident synthesized scans and window sums: they depend only on (map, hypotheses,
    # sensor), which a deployment keeps while the real scans change, so after the first step no ray is cast.
    # Reported beside the step above, not in place of it.
    ctx = relo.Relo(n_orient=360, topk=1024, batch=1024, local_topk=20, early_stop=0, stream=stream,
                    scan_cache_bytes=32 << 30)
    ctx.set_tuning(entries)
    items2 = []
    for it, (g, h, z) in zip(ins, zip(keep[0::3], keep[1::3], keep[2::3])):
        mid = ctx.load_map_dev(g, it.res)
        ctx.set_hypotheses_cells_dev(mid, h)
        items2.append((mid, z, it.angles, it.max_range, it.topk))

    def two():
        ctx.relocalize_batch_dev(items2, res_t)
    for _ in range(3):
        two()
    torch.cuda.synchronize()
    raw2 = bytes(res_t.cpu().numpy())
    same = raw2 == raw
    tab_ms = []
    for i in range(n_steps):
        flush.fill_(i & 0xFF)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        two()
        b_.record(stream)
        b_.synchronize()
        tab_ms.append(a.elapsed_time(b_))
    tables = ctx.scan_cache_stats()
    ctx.close()
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_steps, "warmup": args.warmup,
        "ms_per_step": t_max / n_steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": "synthetic (seeded office/warehouse maps, free-space hypotheses, noisy scans)",
        "config": {"workload": "batched: 64 independent relocalizations per step (map sides 512-2048, beams "
                               "541/720/1081/1440, FoV 180-360 deg, 1k-20k hypotheses, 360 orientations, TAM on the "
                               "top 256 or 1024), one launch per stage; maps resident (EDT at load)",
                   "requests": len(items), "evals_per_step": evals,
                   "hypotheses": int(sum(len(i.hyps) for i in ins)),
                   "l2": "flushed before every timed step (256 MiB write)", "parallelism": f"replicas x{world}"},
        "relocalizations_per_s": world * len(items) * n_steps / (t_max / 1e3),
        "latency_ms": {"p50": pct[len(pct) // 2], "p99": pct[min(len(pct) - 1, int(math.ceil(0.99 * len(pct))) - 1)]},
        "gpu_launches": int(k1 - k0),
        "stage_ms_per_step": {k: round(v / n_steps, 5) for k, v in stage_ms.items()},
        "clocks": clk,
        "launch_shapes": {"tuned_entries": len(entries),
                          "source": os.path.relpath(cache, ROOT) if entries else None,
                          "ms_per_step_builtin": statistics.median(builtin_ms),
                          "ms_per_step_tuned": statistics.median(per),
                          "tuning_run": tuned_info},
        "resident_tables": {"ms_per_step": statistics.median(tab_ms),
                            "relocalizations_per_s": len(items) / (statistics.median(tab_ms) / 1e3),
                            "results_equal": same, "tables": tables},
    }


def run_served(args, world, rank, local, dist):
    """Poisson arrivals against 8 resident maps, p50 / p99 latency per arrival
    rate, for four ways of serving the same requests:

    plain           one request at a time (relo_relocalize), rays cast per request
    plain_tables    one request at a time, synthesized scans and window sums read
                    from the resident per-map tables (scan_cache_bytes)
    served_cast     continuous batching (relo_serve_start / submit / poll), rays cast
    served          continuous batching with the resident tables

    Every mode first runs each pooled request once (sensor plans, kernels and,
    with tables, the tables themselves are then resident: steady state).  The
    rate ladder (unless --rates is given) starts at 250/s and grows by 1.5x
    until p99 passes 50 ms, then bisects the last step twice; the best rate of
    a mode is the highest throughput measured with p99 <= 50 ms.  Each served
    result is compared with the same request run alone (pose agreement)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    maps = workloads.served_maps()
    pool = workloads.served_scans(maps)
    table_bytes = 16 << 30
    P99 = 50.0

    def make_ctx(tables):
        ctx = relo.Relo(n_orient=360, topk=256, batch=200, local_topk=20, early_stop=1, tau=0.95, stream="private",
                        scan_cache_bytes=table_bytes if tables else 0)
        mids = []
        for grid, res, hyps in maps:
            mid = ctx.load_map(grid, res)
            ctx.set_hypotheses(mid, workloads.cell_centres(hyps, res))
            mids.append(mid)
        reqs = [(mids[mi], z, a, mr) for (mi, z, a, mr) in pool]
        results = [ctx.relocalize(*r).as_dict() for r in reqs]   # warm plans, kernels, tables
        return ctx, reqs, results

    def arrivals(rate, seed):
        rng = np.random.default_rng(seed)
        n = max(1, int(rate * args.duration))
        return np.cumsum(rng.exponential(1.0 / rate, size=n)), rng.integers(len(pool), size=n)

    def stats(lat, span, agree=None):
        lat = np.sort(np.asarray(lat))
        out = {"throughput": len(lat) / span, "p50_ms": float(1e3 * lat[len(lat) // 2]),
               "p99_ms": float(1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]), "n": int(len(lat))}
        if agree is not None:
            out["pose_agreement"] = float(np.mean(agree)) if agree else None
        return out

    def run_plain(ctx, reqs, rate, seed):
        t_arr, which = arrivals(rate, seed)
        lat = []
        t0 = time.perf_counter()
        for ta, w in zip(t_arr, which):
            now = time.perf_counter() - t0
            if now < ta:
                time.sleep(ta - now)
            ctx.relocalize(*reqs[w])
            lat.append(time.perf_counter() - t0 - ta)
        return stats(lat, time.perf_counter() - t0)

    def run_srv(ctx, reqs, rate, seed):
        t_arr, which = arrivals(rate, seed)
        lat, pending, agree = [], [], []
        t0 = time.perf_counter()
        i = 0
        while i < len(t_arr) or pending:
            now = time.perf_counter() - t0
            while i < len(t_arr) and t_arr[i] <= now:
                pending.append((ctx.submit(*reqs[which[i]]), which[i]))
                i += 1
            still = []
            for tk, w in pending:
                r = ctx.poll(tk)
                if r is None:
                    still.append((tk, w))
                else:
                    assert r[0] == relo.OK, r[0]
                    lat.append(r[2])
                    agree.append(r[1].as_dict() == alone[w])
            pending = still
            if i < len(t_arr) and not pending:
                time.sleep(max(0.0, min(t_arr[i] - (time.perf_counter() - t0), 0.0005)))
        return stats(lat, time.perf_counter() - t0, agree)

    def ladder(run):
        tab = {}
        if args.rates:
            for k, rate in enumerate(float(x) for x in args.rates.split(",")):
                tab[rate] = run(rate, 4242 + k)
                if tab[rate]["p99_ms"] > 1000.0:
                    break
            return dict(sorted(tab.items()))
        rate, k = 250.0, 0
        while True:
            tab[rate] = run(rate, 4242 + k)
            k += 1
            if tab[rate]["p99_ms"] > P99 or rate > 60000:
                break
            rate = round(rate * 1.5, 1)
        ok = [r for r in tab if tab[r]["p99_ms"] <= P99]
        lo, hi = (max(ok) if ok else 0.0), rate
        for _ in range(2):
            mid = round(0.5 * (lo + hi), 1)
            if mid <= 0:
                break
            tab[mid] = run(mid, 5242 + k)
            k += 1
            if tab[mid]["p99_ms"] <= P99:
                lo = mid
            else:
                hi = mid
        return dict(sorted(tab.items()))

    out = {}
    alone = None
    tables_info = None
    serve_cfgs = [tuple(int(v) for v in c.split("x")) for c in args.serve_configs.split(",")]
    modes = [("plain", False, None), ("plain_tables", True, None), ("served_cast", False, serve_cfgs[0])]
    modes += [("served" if j == 0 else f"served_{b}x{f}", True, (b, f)) for j, (b, f) in enumerate(serve_cfgs)]
    for mode, tables, cfg in modes:
        ctx, reqs, results = make_ctx(tables)
        if alone is None:
            alone = results
        assert results == alone, "resident tables changed a result"
        if cfg is not None:
            ctx.serve_start(max_batch=cfg[0], max_inflight=cfg[1], hbm_budget=8 << 30)
            tab = ladder(lambda rate, seed: run_srv(ctx, reqs, rate, seed))
            ctx.serve_stop()
        else:
            tab = ladder(lambda rate, seed: run_plain(ctx, reqs, rate, seed))
            # device time per stage for one pass over the pool, one request at a time
            ctx.stage_times(reset=True)
            ctx.set_profiling(True)
            for r in reqs:
                ctx.relocalize(*r)
            ms, _, _ = ctx.stage_times(reset=True)
            ctx.set_profiling(False)
            out[mode + "_stage_ms_per_request"] = {k: round(v / len(reqs), 5) for k, v in ms.items()}
        if tables:
            tables_info = ctx.scan_cache_stats()
        out[mode] = {str(k): v for k, v in tab.items()}
        ctx.close()
        torch.cuda.synchronize()

    def best(tab):
        ok = [v["throughput"] for v in tab.values() if v["p99_ms"] <= P99]
        return max(ok) if ok else 0.0

    names = [m for m, _, _ in modes]
    bests = {m: best(out[m]) for m in names}
    agreement = {}
    for m, _, cfg in modes:
        if cfg is not None:
            vals = [(v["pose_agreement"], v["n"]) for v in out[m].values() if v.get("pose_agreement") is not None]
            agreement[m] = sum(a * n for a, n in vals) / max(sum(n for _, n in vals), 1) if vals else None

    def ratio(a, b):
        return round(bests[a] / bests[b], 3) if bests[b] > 0 else None
    return {
        "metric": METRIC, "value": bests["served"], "unit": "relocalizations/s", "n_gpus": world,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": "synthetic (8 resident maps 512^2..4096^2, pooled noisy scans, Poisson arrivals)",
        "config": {"workload": "served: 8 resident maps (two each of 512^2, 1024^2, 2048^2, 4096^2; 1250/5000/10000/"
                               "20000 hypotheses), Poisson arrivals, beams 541/720/1081/1440, 360 orientations, TAM "
                               "in batches of 200 of the top 256 with tau 0.95; continuous batching (max batch x "
                               f"batches in flight {args.serve_configs}, 8 GiB admission budget, 16 GiB of resident "
                               "synthesized scans and window tables) vs one request at a time",
                   "parallelism": "1 GPU"},
        "seconds_per_rate": args.duration,
        "modes": names,
        **out,
        "scan_tables": tables_info,
        "pool": {"requests": len(pool),
                 "tam_batches_mean": float(np.mean([r["n_batches"] for r in alone])),
                 "early_stopped_fraction": float(np.mean([r["n_batches"] < -(-256 // 200) for r in alone]))},
        "pose_agreement": agreement,
        "best_rate_p99_le_50ms": {**{m: round(v, 1) for m, v in bests.items()},
                                  "ratio_served_vs_plain": ratio("served", "plain"),
                                  "ratio_served_vs_plain_tables": ratio("served", "plain_tables"),
                                  "ratio_served_cast_vs_plain": ratio("served_cast", "plain")},
    }


def main():
    faulthandler.enable()
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "ours" and args.workload != "single":
        dist = dist_init(world)
        fn = {"batched": run_batched, "served": run_served, "sweep": run_sweep, "rrt": run_rrt,
              "table2": run_table2, "table3": run_table3}[args.workload]
        line = fn(args, world, rank, local, dist)
        if rank == 0:
            print(json.dumps(line))
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.impl == "reference":
        line = run_reference(args, world, rank)
        if line is not None:
            print(json.dumps(line))
        return
    dist = dist_init(world)
    line = run_ours(args, world, rank, local, dist)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
