#!/usr/bin/env python3
"""Benchmark of the relocalization scoring path on GB300.

One step = one pass of the whole path over the office workload (1024x1024
grid at 0.05 m, 5000 RRT hypotheses, 1081-beam 270-degree noisy scan, 360
orientations, TAM on the SMAD top 256): EDT map precompute, scan
preparation, ray cast + SMAD for every hypothesis, SMAD top-K, batched TAM
over every orientation of every survivor, orientation argmax, local top-k.

value: hypothesis x orientation evaluations (SMAD + TAM) per second with all
inputs resident in HBM; each step is timed with CUDA events on the library's
stream and L2 is flushed (256 MiB write) before every timed step.
e2e: the same metric through the host entry points (relo_update_map,
relo_set_hypotheses, relo_relocalize) from pinned host buffers, host<->device
copies included, wall-clock per step.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload, scaled to the same metric.
"""
from __future__ import annotations

import argparse
import faulthandler
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

METRIC = "hypothesis×orientation evals/s (SMAD+TAM); relocalizations/s at p99 latency"
UNIT = "evals/s"
ROOFLINE_STAGES = ["raycast", "smad", "tam"]   # kernels timed inside the timed region for their roofline
CONFIG_INDEX = 1
WORKLOAD = ("office 1024x1024 @0.05 m, 5000 RRT hypotheses x 360 orientations, 1081-beam 270-deg noisy scan "
            "(N_s 1440), TAM on SMAD top 256 (all batches scored)")
OPS_PER_DDA_STEP = 13     # integer operations of one DDA cell step: the unit of the ray cast's ALU roofline
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="e2e steps (default: min(steps, 200))")
    ap.add_argument("--workload", default="office", choices=["office", "batched", "served", "sweep", "rrt", "table2"],
                    help="office: one request (default); batched: 64 mixed requests per step; "
                         "served: Poisson arrivals against 8 resident maps")
    ap.add_argument("--rates", default="200,400,600,800,1000,1500,2000,3000,4000,5000,6000,7000,8000,10000,12000",
                    help="served: arrival rates per second")
    ap.add_argument("--duration", type=float, default=2.0, help="served: seconds of arrivals per rate")
    ap.add_argument("--coarse", default="smad", choices=["smad", "caer", "smad_direct"],
                    help="office workload: ranking metric, SMAD (Eq. 19-20), CAER (Eq. 21) or SMAD by direct "
                         "window sums (the Table II ablation without prefix sums); the rooflines assume SMAD")
    ap.add_argument("--fine", default="tam", choices=["tam", "tam_mean", "baseline", "lf"],
                    help="office workload: scoring metric, TAM (Eq. 31), TAM_mean (Eq. 34), wp_baseline (Eq. 33) "
                         "or wp_LF (Eq. 32)")
    ap.add_argument("--icp-iters", type=int, default=0,
                    help="office workload: ICP iterations per local top-k pose before its re-evaluation (0: none)")
    ap.add_argument("--serve-configs", default="8x2,16x3,64x3",
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


def committed_traffic(stage: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source
    is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(stage)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2511_01219_gb300", "csrc", rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["dram_bytes_per_launch"] if h == rec["source_sha"] else None


def run_ours(args, world, rank, local, dist):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    wl = workloads.config(CONFIG_INDEX)
    stream = torch.cuda.Stream()
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

    def step():
        ctx.update_map_dev(mid, grid_d)
        ctx.relocalize_dev(mid, z_d, wl.angles, wl.max_range, res_d)

    for _ in range(max(args.warmup, 3)):
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
    bd_total = sum(bd_ms.values())
    shares = {k: v / bd_total for k, v in bd_ms.items()}
    dominant = max(bd_ms, key=bd_ms.get)
    tam_bytes = 2.0 * n_valid * K * n_orient * args.steps          # 2 B field read per valid beam per (h, m)
    roof = {}
    if stage_ms["tam"] > 0:
        gbs = tam_bytes / (stage_ms["tam"] / 1e3) / 1e9
        roof["tam"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": round(gbs / peaks["hbm_gbs"], 4),
                       # the counters were taken with TAM scoring; the other metrics run another epilogue
                       "traffic": committed_traffic("tam") if args.fine == "tam" else None,
                       "peak_source": f"{peak_kind} hbm_gbs",
                       "avg_launch_ms": round(stage_ms["tam"] / max(stage_n["tam"], 1), 4)}
    dda = info[8]
    if stage_ms["raycast"] > 0 and dda:
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        peak_tops = 128 * sm_count * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ops = dda * OPS_PER_DDA_STEP * args.steps
        tops = ops / (stage_ms["raycast"] / 1e3) / 1e12
        roof["raycast"] = {"bound": "alu", "achieved": round(tops, 3), "peak": round(peak_tops, 2),
                           "unit": "Tops/s", "frac": round(tops / peak_tops, 4),
                           "traffic": committed_traffic("raycast"),
                           "peak_source": f"128 int32 lanes x {sm_count} SMs x {peaks.get('sm_max_mhz')} MHz",
                           "dda_steps_per_step": dda,
                           "avg_launch_ms": round(stage_ms["raycast"] / max(stage_n["raycast"], 1), 4)}
    if stage_ms["smad"] > 0:
        smad_bytes = 4.0 * info[0] * info[9] * args.steps          # one Q16 range per (hypothesis, direction)
        gbs = smad_bytes / (stage_ms["smad"] / 1e3) / 1e9
        roof["smad"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": round(gbs / peaks["hbm_gbs"], 4),
                        # the counters are the prefix-sum SMAD kernel's; other rankings run other code
                        "traffic": committed_traffic("smad") if args.coarse == "smad" else None,
                        "peak_source": f"{peak_kind} hbm_gbs",
                        "avg_launch_ms": round(stage_ms["smad"] / max(stage_n["smad"], 1), 4)}
    main_roof = roof.get(dominant) or roof.get("tam")
    pct = sorted(per_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": "synthetic (seeded office map, RRT hypotheses, noisy LiDAR scan)",
        "config": {"workload": WORKLOAD, "map": list(wl.grid.shape), "n_hyp": len(wl.hyps),
                   "n_orient": wl.n_orient, "n_beams": len(wl.ranges), "n_s": wl.n_s, "topk": wl.topk,
                   "evals_per_step": evals_per_step, "l2": "flushed before every timed step (256 MiB write)",
                   "ranking": args.coarse, "scoring": args.fine, "icp_iters": args.icp_iters,
                   "parallelism": f"replicas x{world}"},
        "relocalizations_per_s": world * args.steps / (t_max / 1e3),
        "latency_ms": {"p50": pct[len(pct) // 2], "p99": pct[min(len(pct) - 1, int(math.ceil(0.99 * len(pct))) - 1)]},
        "gpu_launches": int(launches),
        "stage_ms_per_step": {k: round(v / n_bd, 5) for k, v in bd_ms.items()},
        "stage_share": {k: round(v, 4) for k, v in shares.items()},
        "stage_times": f"stage_ms_per_step and stage_share from {n_bd} further steps with every kernel bracketed by "
                       f"events; the timed steps bracket only {', '.join(ROOFLINE_STAGES)} (the roofline kernels)",
        "dominant_kernel": dominant,
        "roofline": main_roof,
        "roofline_all": roof,
        "clocks": clk,
    }
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, ctx, mid, wl, relo, torch, flush, dist, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    ctx.close()
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

def oracle_sample(wl, n_smad: int, n_tam_hyp: int, threads: int):
    """Times the oracle on a bounded sample and scales to the full workload.

    Phases: EDT of the whole map; SMAD of n_smad hypotheses; TAM of the
    first n_tam_hyp hypotheses (standing in for as many survivors: the cost
    does not depend on which) x all orientations.  Returns (evals/s of the
    full workload, estimated seconds per full step, description)."""
    import numpy as np

    import oracle
    prm = oracle.Params(n_orient=wl.n_orient, topk=wl.topk)
    t0 = time.perf_counter()
    d2 = oracle.edt(wl.grid, threads)
    t_edt = time.perf_counter() - t0
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    sel = np.arange(0, len(wl.hyps), max(1, len(wl.hyps) // n_smad))[:n_smad]
    t0 = time.perf_counter()
    oracle.smad(wl.grid, wl.hyps[sel], pl, threads)
    t_smad = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.tam_grid(wl.grid, wl.hyps, np.arange(n_tam_hyp), pl, prm, wl.res, d2, threads)
    t_tam = time.perf_counter() - t0
    n_m = 1 if pl["panoramic"] else pl["n_orient"]
    K = min(wl.topk, len(wl.hyps))
    est = t_edt + t_smad * len(wl.hyps) / len(sel) + t_tam * K / n_tam_hyp
    evals = len(wl.hyps) * n_m + K * pl["n_orient"]
    desc = (f"EDT of the full map + SMAD of {len(sel)}/{len(wl.hyps)} hypotheses + TAM of {n_tam_hyp} hypotheses "
            f"(for {K} survivors) x {pl['n_orient']} orientations, scaled to the full step")
    return evals / est, est, desc


def cpu_baseline(wl):
    """The oracle on all host cores, and on one core (a smaller sample)."""
    import oracle
    threads = oracle.max_threads()
    v, est, desc = oracle_sample(wl, n_smad=len(wl.hyps), n_tam_hyp=min(wl.topk, len(wl.hyps)), threads=threads)
    v1, est1, desc1 = oracle_sample(wl, n_smad=100, n_tam_hyp=4, threads=1)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
            "est_s_per_step": est,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": desc1, "est_s_per_step": est1}}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import oracle
    import workloads
    oracle.build()
    wl = workloads.config(CONFIG_INDEX)
    threads = oracle.max_threads()
    for _ in range(max(args.warmup, 0)):
        oracle_sample(wl, 100, 2, threads)
    vals, ests = [], []
    desc = ""
    for _ in range(args.steps):
        v, est, desc = oracle_sample(wl, 100, 2, threads)
        vals.append(v)
        ests.append(est)
    total = sum(ests)
    value = len(ests) / total * (vals[0] * ests[0])    # evals per step / mean seconds per step
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ests), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded office map, RRT hypotheses, noisy LiDAR scan)",
        "config": {"workload": WORKLOAD, "parallelism": "host cores"},
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
    wl = workloads.config(CONFIG_INDEX)
    gx, gy, gth = wl.gt_pose
    cx, cy = int(round(gx / wl.res - 0.5)), int(round(gy / wl.res - 0.5))
    step = int(round(0.1 / wl.res))
    offs = np.arange(-7, 8) * step
    free = wl.grid < 65
    axis = None
    for ax, (dx, dy) in enumerate(((1, 0), (0, 1))):
        cells = np.stack([cx + dx * offs, cy + dy * offs], 1)
        inside = (cells[:, 0] >= 0) & (cells[:, 0] < wl.grid.shape[1]) & (cells[:, 1] >= 0) & (cells[:, 1] < wl.grid.shape[0])
        if inside.all() and free[cells[:, 1], cells[:, 0]].all():
            axis = "xy"[ax]
            break
    if axis is None:
        raise RuntimeError("no axis through the true position with 15 free cells")
    n_s = wl.n_s
    m_true = int(round(gth / (2 * math.pi) * n_s)) % n_s
    q_true = m_true // (n_s // 360)
    sweep_q = [(q_true + 10 * j) % 360 for j in range(36)]   # 10-degree steps from the true orientation
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
    wl = workloads.config(CONFIG_INDEX)
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
    wl = workloads.config(CONFIG_INDEX)
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


def run_batched(args, world, rank, local, dist):
    """64 independent relocalizations per step (mixed map sizes, beam counts,
    FoVs and hypothesis counts), one launch per stage, all inputs resident."""
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
    for _ in range(max(args.warmup, 3)):
        ctx.relocalize_batch_dev(items, res_t)
    torch.cuda.synchronize()
    raw = bytes(res_t.cpu().numpy())
    results = [relo.result_from_bytes(raw[i * relo.RESULT_BYTES:(i + 1) * relo.RESULT_BYTES]) for i in range(len(items))]
    assert all(r.status == relo.OK for r in results), [r.status for r in results]
    evals = sum(int(r.n_smad_evals + r.n_tam_evals) for r in results)
    ctx.set_profiling(True)
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
        ctx.relocalize_batch_dev(items, res_t)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(dist)
    per = [a.elapsed_time(b) for a, b in ev]
    total = sum(per)
    stage_ms, stage_n, k1 = ctx.stage_times(reset=True)
    t_max = max_over_ranks(dist, total)
    value = sum_over_ranks(dist, float(evals * args.steps)) / (t_max / 1e3)
    pct = sorted(per)
    ctx.close()
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": "synthetic (seeded office/warehouse maps, free-space hypotheses, noisy scans)",
        "config": {"workload": "batched: 64 independent relocalizations per step (map sides 512-2048, beams "
                               "541/720/1081/1440, FoV 180-360 deg, 1k-20k hypotheses, 360 orientations, TAM on the "
                               "top 256 or 1024), one launch per stage; maps resident (EDT at load)",
                   "requests": len(items), "evals_per_step": evals,
                   "hypotheses": int(sum(len(i.hyps) for i in ins)),
                   "l2": "flushed before every timed step (256 MiB write)", "parallelism": f"replicas x{world}"},
        "relocalizations_per_s": world * len(items) * args.steps / (t_max / 1e3),
        "latency_ms": {"p50": pct[len(pct) // 2], "p99": pct[min(len(pct) - 1, int(math.ceil(0.99 * len(pct))) - 1)]},
        "gpu_launches": int(k1 - k0),
        "stage_ms_per_step": {k: round(v / args.steps, 5) for k, v in stage_ms.items()},
        "clocks": clk,
    }


def run_served(args, world, rank, local, dist):
    """Poisson arrivals against 8 resident maps, p50 / p99 latency per arrival
    rate, for four ways of serving the same requests:

    plain           one request at a time (relo_relocalize), rays cast per request
    plain_tables    one request at a time, synthesized scans read from the
                    resident per-map tables (scan_cache_bytes)
    served_cast     continuous batching (relo_serve_start / submit / poll), rays cast
    served          continuous batching with the resident tables

    Every mode first runs each pooled request once (sensor plans, kernels and,
    with tables, the tables themselves are then resident: steady state).  A
    mode's rate ladder stops once its p99 passes 1 s (it is saturated)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    import workloads

    torch.cuda.set_device(local)
    maps = workloads.served_maps()
    pool = workloads.served_scans(maps)
    rates = [float(x) for x in args.rates.split(",")]
    table_bytes = 16 << 30

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

    def stats(lat, span):
        lat = np.sort(np.asarray(lat))
        return {"throughput": len(lat) / span, "p50_ms": float(1e3 * lat[len(lat) // 2]),
                "p99_ms": float(1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]), "n": int(len(lat))}

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

    def run_srv(ctx, reqs, rate, seed, agree):
        t_arr, which = arrivals(rate, seed)
        lat, pending = [], []
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
        return stats(lat, time.perf_counter() - t0)

    out = {}
    alone = None
    tables_info = None
    serve_cfgs = [tuple(int(v) for v in c.split("x")) for c in args.serve_configs.split(",")]
    modes = [("plain", False, None), ("plain_tables", True, None), ("served_cast", False, max(serve_cfgs))]
    modes += [(f"served_{b}x{f}", True, (b, f)) for (b, f) in serve_cfgs]
    for mode, tables, cfg in modes:
        ctx, reqs, results = make_ctx(tables)
        if alone is None:
            alone = results
        assert results == alone, "resident tables changed a result"
        agree = []
        tab = {}
        if cfg is not None:
            ctx.serve_start(max_batch=cfg[0], max_inflight=cfg[1], hbm_budget=8 << 30)
        run = (lambda rate, seed: run_srv(ctx, reqs, rate, seed, agree)) if cfg is not None else \
            (lambda rate, seed: run_plain(ctx, reqs, rate, seed))
        for k, rate in enumerate(rates):
            tab[rate] = run(rate, 4242 + k)
            if tab[rate]["p99_ms"] > 1000.0:
                break
        # refine between the fastest rate that kept p99 <= 50 ms and the next one tried
        ok = [r for r in tab if tab[r]["p99_ms"] <= 50.0]
        above = [r for r in tab if ok and r > max(ok)]
        if ok and above:
            lo, hi = max(ok), min(above)
            for k, f in enumerate((0.25, 0.5, 0.75)):
                rate = round(lo + f * (hi - lo), 1)
                tab[rate] = run(rate, 5242 + k)
        tab = dict(sorted(tab.items()))
        if cfg is not None:
            ctx.serve_stop()
            out[mode + "_pose_agreement"] = float(np.mean(agree)) if agree else None
        if tables:
            tables_info = ctx.scan_cache_stats()
        if cfg is None:
            # device time per stage for one pass over the pool, one request at a time
            ctx.stage_times(reset=True)
            ctx.set_profiling(True)
            for r in reqs:
                ctx.relocalize(*r)
            ms, _, _ = ctx.stage_times(reset=True)
            ctx.set_profiling(False)
            out[mode + "_stage_ms_per_request"] = {k: round(v / len(reqs), 5) for k, v in ms.items()}
        out[mode] = {str(k): v for k, v in tab.items()}
        ctx.close()
        torch.cuda.synchronize()

    def best(tab, cap=None):
        ok = [v["throughput"] for k, v in tab.items() if v["p99_ms"] <= 50.0 and (cap is None or float(k) <= cap)]
        return max(ok) if ok else 0.0
    bests = {m: best(out[m]) for m, _, _ in modes}
    bests_cfg = {m: best(out[m], 2000.0) for m in bests}
    served_modes = [m for m, t, c in modes if t and c is not None]
    best_served = max(served_modes, key=lambda m: bests[m])
    bests["served"] = bests[best_served]
    b_srv, b_pln = bests["served"], bests["plain"]
    return {
        "metric": METRIC, "value": b_srv, "unit": "relocalizations/s", "n_gpus": world, "steps": len(rates),
        "warmup": len(pool), "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32/i64+f32", "data": "synthetic (8 resident maps 512^2..4096^2, pooled noisy scans, Poisson arrivals)",
        "config": {"workload": "served: 8 resident maps (two each of 512^2, 1024^2, 2048^2, 4096^2; 1250/5000/10000/"
                               "20000 hypotheses), Poisson arrivals, beams 541/720/1081/1440, 360 orientations, TAM "
                               "in batches of 200 of the top 256 with tau 0.95; continuous batching (max batch x "
                               "batches in flight as listed, 8 GiB admission budget, 16 GiB of resident synthesized "
                               "scans and window tables) vs one request at a time",
                   "rates_per_s": rates, "seconds_per_rate": args.duration, "parallelism": "1 GPU"},
        **out,
        "scan_tables": tables_info,
        "pool": {"requests": len(pool),
                 "tam_batches_mean": float(np.mean([r["n_batches"] for r in alone])),
                 "early_stopped_fraction": float(np.mean([r["n_batches"] < -(-256 // 200) for r in alone]))},
        "best_served_config": best_served,
        "best_rate_p99_le_50ms": {**bests, "ratio_served_vs_plain": (b_srv / b_pln) if b_pln > 0 else None,
                                  "ratio_served_vs_plain_tables": (b_srv / bests["plain_tables"])
                                  if bests["plain_tables"] > 0 else None},
        "best_rate_p99_le_50ms_rates_le_2000": bests_cfg,
    }


def main():
    faulthandler.enable()
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "ours" and args.workload != "office":
        dist = dist_init(world)
        fn = {"batched": run_batched, "served": run_served, "sweep": run_sweep, "rrt": run_rrt,
              "table2": run_table2}[args.workload]
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
