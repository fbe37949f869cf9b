"""Autotuner of the batched stages' launch shapes (relo_set_tuning).

The library picks the launch shapes of its stage kernels by rule: TAM takes
survivors in tasks of one band phase (a chunk of up to 64), the ray cast and
TAM fill every resident CTA slot.  Which shape is fastest depends on the
request shapes (beam count, orientations, K) and on the GPU, so this module
measures: for the ray cast it tries CTAs per SM, and for every TAM shape
bucket (values-per-lane class, n_orient, K) present in a workload it tries
chunk sizes and CTAs per SM, one bucket at a time (the others at their best
so far), timing the stage with the library's own CUDA events over a few
repetitions of the workload.  Shapes never change results, only time.

A workload of single requests is tuned apart (``single``): one request's TAM
tasks alone fill the GPU, so its best shape differs from a mixed batch's.

The result is a list of tuning entries, cached in a JSON file per device
(``tuning/<device>.json`` next to this module) and loaded into a context with
``Relo.set_tuning(load(path))``.
"""
from __future__ import annotations

import json
import os
import statistics
import time

from . import TUNE_CAST, TUNE_TAM, TUNE_TAM_ONE, tam_class

HERE = os.path.dirname(os.path.abspath(__file__))
CHUNKS = (8, 16, 24, 32, 48, 64)
TAM_CTAS = (0, 4, 3)          # resident CTAs per SM (0: all that fit)
CAST_CTAS = (0, 5, 4, 3)


def cache_path(device_name: str) -> str:
    safe = "".join(c if c.isalnum() else "_" for c in device_name).strip("_")
    return os.path.join(HERE, "tuning", f"{safe}.json")


def load(path: str) -> list:
    """Tuning entries [(kind, key, val)] from a cache file ([] if it is missing)."""
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return []
    return [(e["kind"], tuple(e["key"]), tuple(e["val"])) for e in rec.get("entries", [])]


def save(path: str, entries: list, meta: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    rec = {**meta, "entries": [{"kind": k, "key": list(key), "val": list(val)} for k, key, val in entries]}
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(rec, f, indent=1)
    os.replace(tmp, path)


def buckets(shapes) -> list:
    """TAM shape buckets (class, n_orient, K) of request shapes [(n_beams, n_orient, K)], sorted."""
    return sorted({(tam_class(nb), no, k) for nb, no, k in shapes})


def stage_ms(ctx, run, stage: str, reps: int) -> float:
    """Median device time of one stage over reps runs of the workload (the library's events)."""
    import torch
    ctx.set_profiling(True)
    vals = []
    for _ in range(reps):
        ctx.stage_times(reset=True)
        run()
        ms, _, _ = ctx.stage_times(reset=True)
        vals.append(ms[stage])
    ctx.set_profiling(False)
    torch.cuda.synchronize()
    return statistics.median(vals)


def tune(ctx, run, shapes, reps: int = 3, log=None, single: bool = False) -> dict:
    """Measured search.  run(): one pass of the workload on ctx; shapes: its
    requests' (n_beams after the beam stride, n_orient, K).  With single, run()
    issues one request per launch: the TAM entries are then RELO_TUNE_TAM_ONE
    (launches of a single request look them up first) and the ray cast is left
    to the batched tuning.  Returns {"entries": [...], "cast_ms": (built-in,
    tuned), "tam_ms": (built-in, tuned), "trials": [...]}; ctx is left with the
    tuned entries set."""
    t0 = time.time()
    trials = []
    tam_kind = TUNE_TAM_ONE if single else TUNE_TAM
    ctx.set_tuning([])
    run()
    base_tam = stage_ms(ctx, run, "tam", reps)
    base_cast = stage_ms(ctx, run, "raycast", reps)
    trials.append({"entries": [], "tam_ms": base_tam, "raycast_ms": base_cast})
    best_cast, best_cast_ms = None, base_cast
    for c in (() if single else CAST_CTAS[1:]):
        e = [(TUNE_CAST, (0, 0, 0), (c, 0))]
        ctx.set_tuning(e)
        ms = stage_ms(ctx, run, "raycast", reps)
        trials.append({"entries": e, "raycast_ms": ms})
        if ms < best_cast_ms:
            best_cast, best_cast_ms = e[0], ms
    chosen = {}
    best_tam_ms = base_tam
    for b in buckets(shapes):
        for chunk in CHUNKS:
            for cps in TAM_CTAS:
                cand = dict(chosen)
                cand[b] = (chunk, cps)
                e = [(tam_kind, k, v) for k, v in cand.items()]
                ctx.set_tuning(e)
                ms = stage_ms(ctx, run, "tam", reps)
                trials.append({"entries": e, "tam_ms": ms})
                if ms < best_tam_ms:
                    best_tam_ms = ms
                    chosen = cand
        if log:
            log(f"bucket {b}: {chosen.get(b)} tam {best_tam_ms:.4f} ms ({time.time() - t0:.0f} s)")
    entries = [(tam_kind, k, v) for k, v in chosen.items()] + ([best_cast] if best_cast else [])
    ctx.set_tuning(entries)
    return {"entries": entries, "tam_ms": (base_tam, best_tam_ms), "cast_ms": (base_cast, best_cast_ms),
            "trials": trials, "seconds": time.time() - t0}
