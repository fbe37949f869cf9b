"""GB300 relocalization scoring: Python binding of the C ABI in include/relo.h.

This module only marshals arguments: every step of the scoring path runs in
the CUDA kernels of ``librelo.so`` (built in-tree for sm_103a by
``paper_2511_01219_gb300._build.build()``).  PyTorch provides device buffers
and streams; there is no CPU fallback, and importing a context without the
compiled library raises.

Entry points mirror the C names: ``Relo.load_map`` (EDT precompute, Sec.
III-A item 3), ``Relo.set_hypotheses`` (Eq. 6), ``Relo.relocalize`` (Eq. 3
via SMAD ranking, Eq. 16-20, and batched TAM, Eq. 22-31).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librelo.so")

OK = 0
PENDING = 1
E_INVALID_ARG = -1
E_BEAM_GRID = -2
E_NO_HYPOTHESES = -3
E_OVER_BUDGET = -4
E_CUDA = -5
E_TIMEOUT = -6
E_NO_VALID_BEAMS = -7
E_NOT_FOUND = -8

STAGE_SMAD_NUM, STAGE_SMAD_M, STAGE_SURVIVORS, STAGE_TAM, STAGE_BEST_M, STAGE_LOCAL_TOPK, STAGE_SCAN_INFO = range(7)
SCAN_INFO_LEN = 10

EXPORTED = [
    "relo_default_params", "relo_create", "relo_destroy", "relo_last_error", "relo_set_params", "relo_load_map",
    "relo_load_map_dev", "relo_update_map", "relo_update_map_dev", "relo_unload_map", "relo_map_tables_dev", "relo_set_hypotheses",
    "relo_set_hypotheses_cells_dev", "relo_relocalize", "relo_relocalize_dev", "relo_get_stage",
    "relo_synth_scans_dev", "relo_set_profiling", "relo_stage_times", "relo_edt_noalloc",
    "relo_relocalize_batch", "relo_relocalize_batch_dev", "relo_serve_start", "relo_submit", "relo_poll",
    "relo_serve_stop", "relo_scan_cache_stats", "relo_set_profiling_mask", "relo_rrt_hypotheses_dev",
    "relo_probe_l2_stream", "relo_probe_l2_gather", "relo_rrt_sample",
    "relo_submit_until", "relo_set_tuning", "relo_tam_class", "relo_map_walk_boxes_dev",
]
STAGES = ["edt", "scan_prep", "raycast", "topk", "tam", "select", "smad", "edt_field"]


class Params(ctypes.Structure):
    _fields_ = [
        ("z_hit", ctypes.c_double), ("sigma_hit", ctypes.c_double), ("z_rand", ctypes.c_double),
        ("eps", ctypes.c_double), ("d_max", ctypes.c_double), ("a_mid_min", ctypes.c_double),
        ("a_mid_max", ctypes.c_double), ("a_low_min", ctypes.c_double), ("a_low_max", ctypes.c_double),
        ("tau", ctypes.c_double), ("panoramic_ratio", ctypes.c_double), ("n_orient", ctypes.c_int32),
        ("topk", ctypes.c_int32), ("batch", ctypes.c_int32), ("local_topk", ctypes.c_int32),
        ("n_skip_beam", ctypes.c_int32), ("early_stop", ctypes.c_int32), ("hbm_budget", ctypes.c_int64),
        ("max_range", ctypes.c_double), ("scan_cache_bytes", ctypes.c_int64), ("ray_tables", ctypes.c_int32),
        ("coarse_metric", ctypes.c_int32), ("fine_metric", ctypes.c_int32), ("icp_iters", ctypes.c_int32),
    ]

COARSE_SMAD, COARSE_CAER, COARSE_SMAD_DIRECT, COARSE_NONE = 0, 1, 2, 3
FINE_TAM, FINE_TAM_MEAN, FINE_BASELINE, FINE_LF = 0, 1, 2, 3
TUNE_TAM, TUNE_CAST, TUNE_TAM_ONE = 1, 2, 3


class TuneEntry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("key", ctypes.c_int32 * 3), ("val", ctypes.c_int32 * 2)]


class Result(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_double), ("y", ctypes.c_double), ("theta", ctypes.c_double), ("tam", ctypes.c_double),
        ("smad", ctypes.c_double), ("smad_num", ctypes.c_int64), ("n_smad_evals", ctypes.c_int64),
        ("n_tam_evals", ctypes.c_int64), ("hyp", ctypes.c_int32), ("m", ctypes.c_int32),
        ("n_batches", ctypes.c_int32), ("status", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


RESULT_BYTES = ctypes.sizeof(Result)


class Request(ctypes.Structure):
    _fields_ = [("map_id", ctypes.c_int32), ("ranges", ctypes.c_void_p), ("angles", ctypes.c_void_p),
                ("n_beams", ctypes.c_int32), ("max_range", ctypes.c_float), ("topk", ctypes.c_int32)]


class ReloError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"relo error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded librelo.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2511_01219_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        sig = {
            "relo_default_params": (None, [P]),
            "relo_create": (ctypes.c_int, [P, P, P]),
            "relo_destroy": (ctypes.c_int, [P]),
            "relo_last_error": (ctypes.c_char_p, [P]),
            "relo_set_params": (ctypes.c_int, [P, P]),
            "relo_load_map": (ctypes.c_int, [P, P, I32, I32, D, D, D, P]),
            "relo_load_map_dev": (ctypes.c_int, [P, P, I32, I32, D, D, D, P]),
            "relo_update_map_dev": (ctypes.c_int, [P, I32, P]),
            "relo_update_map": (ctypes.c_int, [P, I32, P]),
            "relo_unload_map": (ctypes.c_int, [P, I32]),
            "relo_map_tables_dev": (ctypes.c_int, [P, I32, P, P, P]),
            "relo_map_walk_boxes_dev": (ctypes.c_int, [P, I32, P, I64, P]),
            "relo_set_hypotheses": (ctypes.c_int, [P, I32, P, I32]),
            "relo_set_hypotheses_cells_dev": (ctypes.c_int, [P, I32, P, I32]),
            "relo_relocalize": (ctypes.c_int, [P, I32, P, P, I32, F, P]),
            "relo_relocalize_dev": (ctypes.c_int, [P, I32, P, P, I32, F, P]),
            "relo_get_stage": (ctypes.c_int, [P, I32, P, I64]),
            "relo_synth_scans_dev": (ctypes.c_int, [P, I32, P, I32, P, I32, F, P, P, I64, P]),
            "relo_set_profiling": (ctypes.c_int, [P, I32]),
            "relo_set_profiling_mask": (ctypes.c_int, [P, ctypes.c_uint32]),
            "relo_stage_times": (ctypes.c_int, [P, P, P, I32, I32, P]),
            "relo_edt_noalloc": (ctypes.c_int, [P, I32, I32, P, P]),
            "relo_probe_l2_stream": (ctypes.c_int, [P, I64, I32, P, P]),
            "relo_rrt_sample": (ctypes.c_int, [P, P, I32, I32, D, D, D, D, D, D, I32, ctypes.c_uint64, I32, I32, P,
                                               I32, P, P, P, P]),
            "relo_probe_l2_gather": (ctypes.c_int, [P, I32, I64, P, P, P]),
            "relo_relocalize_batch": (ctypes.c_int, [P, P, I32, P]),
            "relo_relocalize_batch_dev": (ctypes.c_int, [P, P, I32, P]),
            "relo_serve_start": (ctypes.c_int, [P, I32, I32, I64]),
            "relo_submit": (ctypes.c_int, [P, I32, P, P, I32, F, P]),
            "relo_submit_until": (ctypes.c_int, [P, I32, P, P, I32, F, D, P]),
            "relo_set_tuning": (ctypes.c_int, [P, P, I32]),
            "relo_tam_class": (ctypes.c_int, [I32]),
            "relo_poll": (ctypes.c_int, [P, I64, P, P]),
            "relo_serve_stop": (ctypes.c_int, [P]),
            "relo_scan_cache_stats": (ctypes.c_int, [P, P, I32]),
            "relo_rrt_hypotheses_dev": (ctypes.c_int, [P, P, I32, I32, D, D, D, D, D, D, I32, ctypes.c_uint64, I32, I32,
                                                       P, I32, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_params(**overrides) -> Params:
    p = Params()
    lib().relo_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _t_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the handle of CUDA's legacy default stream


def _stream_handle(stream):
    """stream: None (torch's current stream), "private" (a new stream owned by
    the context), a torch.cuda.Stream, or a raw cudaStream_t integer."""
    if isinstance(stream, str) and stream == "private":
        return None
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    h = int(getattr(stream, "cuda_stream", stream))
    return ctypes.c_void_p(h if h != 0 else CUDA_STREAM_LEGACY)


class Relo:
    """One library context (maps, hypothesis sets, scratch) on one CUDA stream.

    By default the context runs on torch's current stream, so device tensors
    that torch wrote are ready when the library's kernels read them.
    """

    def __init__(self, params: Params | None = None, stream=None, **overrides):
        self._L = lib()
        p = params if params is not None else default_params(**overrides)
        h = ctypes.c_void_p()
        s = _stream_handle(stream)
        rc = self._L.relo_create(ctypes.byref(p), s, ctypes.byref(h))
        if rc != OK:
            raise ReloError(rc, "relo_create failed")
        self._h = h
        self.params = p

    def _check(self, rc: int, what: str):
        if rc != OK:
            raise ReloError(rc, f"{what}: {self._L.relo_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.relo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: Params):
        self._check(self._L.relo_set_params(self._h, ctypes.byref(params)), "set_params")
        self.params = params

    # ---- maps --------------------------------------------------------------------------
    def load_map(self, grid: np.ndarray, res: float, origin=(0.0, 0.0)) -> int:
        g = np.ascontiguousarray(grid, dtype=np.int8)
        mid = ctypes.c_int32(-1)
        self._check(self._L.relo_load_map(self._h, _np_ptr(g), g.shape[1], g.shape[0], res, origin[0], origin[1],
                                          ctypes.byref(mid)), "load_map")
        return mid.value

    def load_map_dev(self, grid_t, res: float, origin=(0.0, 0.0)) -> int:
        mid = ctypes.c_int32(-1)
        self._check(self._L.relo_load_map_dev(self._h, _t_ptr(grid_t), grid_t.shape[1], grid_t.shape[0], res,
                                              origin[0], origin[1], ctypes.byref(mid)), "load_map_dev")
        return mid.value

    def update_map_dev(self, map_id: int, grid_t):
        self._check(self._L.relo_update_map_dev(self._h, map_id, _t_ptr(grid_t)), "update_map_dev")

    def update_map(self, map_id: int, grid: np.ndarray):
        """Host grid (numpy, or a pinned torch CPU tensor passed as its data pointer via update_map_ptr)."""
        g = np.ascontiguousarray(grid, dtype=np.int8)
        self._check(self._L.relo_update_map(self._h, map_id, _np_ptr(g)), "update_map")

    def update_map_ptr(self, map_id: int, host_ptr: int):
        self._check(self._L.relo_update_map(self._h, map_id, ctypes.c_void_p(host_ptr)), "update_map")

    def set_hypotheses_ptr(self, map_id: int, xy_host_ptr: int, n: int):
        self._check(self._L.relo_set_hypotheses(self._h, map_id, ctypes.c_void_p(xy_host_ptr), n), "set_hypotheses")

    def relocalize_ptr(self, map_id: int, ranges_host_ptr: int, angles: np.ndarray, n: int, max_range: float,
                       out: "Result") -> "Result":
        a = np.ascontiguousarray(angles, dtype=np.float32)
        self._check(self._L.relo_relocalize(self._h, map_id, ctypes.c_void_p(ranges_host_ptr), _np_ptr(a), n,
                                            max_range, ctypes.byref(out)), "relocalize")
        return out

    def unload_map(self, map_id: int):
        self._check(self._L.relo_unload_map(self._h, map_id), "unload_map")

    def map_tables(self, map_id: int, shape):
        """(d2 int32, field uint16 as int32, occ uint8) torch tensors on the current device."""
        import torch
        H, W = shape
        d2 = torch.empty((H, W), dtype=torch.int32, device="cuda")
        fld = torch.empty((H, W), dtype=torch.int16, device="cuda")
        occ = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        self._check(self._L.relo_map_tables_dev(self._h, map_id, _t_ptr(d2), _t_ptr(fld), _t_ptr(occ)),
                    "map_tables")
        return d2, fld.to(torch.int32) & 0xFFFF, occ

    def walk_boxes(self, map_id: int, shape):
        """The ray walk's empty boxes of tiles (relo_map_walk_boxes_dev) as an int32 numpy array
        [4, ceil(H/8) + 1, ceil(W/8) + 1] of the packed uint16 entries."""
        import torch
        H, W = shape
        TW, TH = (W + 7) // 8, (H + 7) // 8
        n = 4 * (TW + 1) * (TH + 1)
        buf = torch.empty(n, dtype=torch.int16, device="cuda")
        got = ctypes.c_int64(0)
        self._check(self._L.relo_map_walk_boxes_dev(self._h, map_id, _t_ptr(buf), n, ctypes.byref(got)), "walk_boxes")
        return (buf.cpu().numpy().view("uint16").astype("int32")).reshape(4, TH + 1, TW + 1)

    # ---- hypotheses ----------------------------------------------------------------------
    def set_hypotheses(self, map_id: int, xy: np.ndarray):
        a = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self._check(self._L.relo_set_hypotheses(self._h, map_id, _np_ptr(a), len(a)), "set_hypotheses")

    def set_hypotheses_cells_dev(self, map_id: int, cells_t):
        self._check(self._L.relo_set_hypotheses_cells_dev(self._h, map_id, _t_ptr(cells_t), cells_t.shape[0]),
                    "set_hypotheses_cells_dev")

    # ---- relocalization ------------------------------------------------------------------
    def relocalize(self, map_id: int, ranges: np.ndarray, angles: np.ndarray, max_range: float) -> Result:
        z = np.ascontiguousarray(ranges, dtype=np.float32)
        a = np.ascontiguousarray(angles, dtype=np.float32)
        out = Result()
        self._check(self._L.relo_relocalize(self._h, map_id, _np_ptr(z), _np_ptr(a), len(z), max_range,
                                            ctypes.byref(out)), "relocalize")
        return out

    def relocalize_dev(self, map_id: int, ranges_t, angles: np.ndarray, max_range: float, result_t):
        """Asynchronous: result_t is a device uint8 tensor of RESULT_BYTES bytes."""
        a = np.ascontiguousarray(angles, dtype=np.float32)
        self._check(self._L.relo_relocalize_dev(self._h, map_id, _t_ptr(ranges_t), _np_ptr(a), int(ranges_t.numel()),
                                                max_range, _t_ptr(result_t)), "relocalize_dev")

    def set_profiling(self, on: bool):
        self._check(self._L.relo_set_profiling(self._h, int(bool(on))), "set_profiling")

    def set_profiling_stages(self, stages):
        """Profile only the named stages (names from STAGES); an empty list turns profiling off."""
        mask = 0
        for name in stages:
            mask |= 1 << STAGES.index(name)
        self._check(self._L.relo_set_profiling_mask(self._h, mask), "set_profiling_mask")

    def stage_times(self, reset: bool = False):
        """({stage: ms}, {stage: launches}, kernels launched since creation)."""
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_int64 * len(STAGES))()
        k = ctypes.c_int64(0)
        self._check(self._L.relo_stage_times(self._h, ms, n, len(STAGES), int(reset), ctypes.byref(k)), "stage_times")
        return dict(zip(STAGES, list(ms))), dict(zip(STAGES, list(n))), k.value

    def scan_info(self) -> list:
        """[N_s, n_orient, n_enum, N_valid, k_retained, sum_real, K, batches, DDA steps, N_h] of the last request."""
        import torch
        t = torch.empty(SCAN_INFO_LEN, dtype=torch.int64, device="cuda")
        self.stage(STAGE_SCAN_INFO, t)
        return t.cpu().tolist()

    def dda_steps(self) -> int:
        return int(self.scan_info()[8])

    def scan_cache_stats(self) -> dict:
        """Resident synthesized scans: tables and bytes held, requests that read a table, requests that cast,
        evictions, window tables held, requests whose SMAD read a window table."""
        v = (ctypes.c_int64 * 7)()
        self._check(self._L.relo_scan_cache_stats(self._h, v, 7), "scan_cache_stats")
        return dict(zip(["tables", "bytes", "hits", "misses", "evictions", "win_tables", "win_hits"], list(v)))

    def rrt_hypotheses(self, clearance_t, res: float, p0, rho: float, eta_max: float = 0.6, r_robot: float = 0.21,
                       eps_gain: int = 2, seed: int = 0, max_rounds: int = 500, node_cap: int = 4_000_000,
                       cap: int = 1_000_000):
        """Algorithm 1 on the GPU (the serial tree for the sampler's random points): (xy float32 [n, 2] metres on
        the device, in node order, rounds, nodes)."""
        import torch
        h, w = clearance_t.shape
        xy = torch.empty((cap, 2), dtype=torch.float32, device=clearance_t.device)
        n, r, nn = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._L.relo_rrt_hypotheses_dev(self._h, _t_ptr(clearance_t), w, h, res, float(p0[0]),
                                                   float(p0[1]), rho, eta_max, r_robot, eps_gain, seed, max_rounds,
                                                   node_cap, _t_ptr(xy), cap, ctypes.byref(n), ctypes.byref(r),
                                                   ctypes.byref(nn)), "rrt_hypotheses")
        return xy[: n.value], r.value, nn.value

    def rrt_sample(self, grid: np.ndarray, res: float, p0, rho: float, eta_max: float = 0.6, r_robot: float = 0.21,
                   eps_gain: int = 2, seed: int = 0, max_rounds: int = 500, node_cap: int = 4_000_000,
                   cap: int = 1_000_000, with_clearance: bool = False):
        """Algorithm 1 from the occupancy grid (host arrays): (xy float64 [n, 2] metres, rounds, nodes[,
        clearance float32 [h, w] metres])."""
        g = np.ascontiguousarray(grid, dtype=np.int8)
        h, w = g.shape
        xy = np.zeros((cap, 2), np.float64)
        clr = np.zeros((h, w), np.float32) if with_clearance else None
        n, r, nn = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._L.relo_rrt_sample(self._h, g.ctypes.data, w, h, res, float(p0[0]), float(p0[1]), rho,
                                            eta_max, r_robot, eps_gain, seed, max_rounds, node_cap, xy.ctypes.data,
                                            cap, ctypes.byref(n), ctypes.byref(r), ctypes.byref(nn),
                                            None if clr is None else clr.ctypes.data), "rrt_sample")
        out = (xy[: n.value].copy(), r.value, nn.value)
        return out + (clr,) if with_clearance else out

    def set_tuning(self, entries):
        """Launch shapes (relo_set_tuning): entries [(kind, (k0, k1, k2), (v0, v1))]; [] clears."""
        arr = (TuneEntry * max(len(entries), 1))()
        for i, (kind, key, val) in enumerate(entries):
            arr[i].kind = kind
            for j in range(3):
                arr[i].key[j] = int(key[j])
            for j in range(2):
                arr[i].val[j] = int(val[j])
        self._check(self._L.relo_set_tuning(self._h, arr, len(entries)), "set_tuning")

    def kernels_launched(self) -> int:
        k = ctypes.c_int64(0)
        self._check(self._L.relo_stage_times(self._h, None, None, 0, 0, ctypes.byref(k)), "stage_times")
        return k.value

    def relocalize_batch(self, items) -> list:
        """items: [(map_id, ranges ndarray, angles ndarray, max_range[, topk])]; blocking; list of Result."""
        keep = []
        arr = (Request * len(items))()
        for i, it in enumerate(items):
            mid, z, a, mr = it[:4]
            z = np.ascontiguousarray(z, dtype=np.float32)
            a = np.ascontiguousarray(a, dtype=np.float32)
            keep += [z, a]
            arr[i] = Request(mid, z.ctypes.data, a.ctypes.data, len(z), mr, it[4] if len(it) > 4 else 0)
        out = (Result * len(items))()
        self._check(self._L.relo_relocalize_batch(self._h, arr, len(items), out), "relocalize_batch")
        return list(out)

    def relocalize_batch_dev(self, items, results_t):
        """items: [(map_id, ranges device tensor, angles ndarray, max_range[, topk])]; asynchronous;
        results_t: device uint8 tensor of len(items) * RESULT_BYTES bytes."""
        keep = []
        arr = (Request * len(items))()
        for i, it in enumerate(items):
            mid, zt, a, mr = it[:4]
            a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
            arr[i] = Request(mid, zt.data_ptr(), a.ctypes.data, int(zt.numel()), mr, it[4] if len(it) > 4 else 0)
        self._check(self._L.relo_relocalize_batch_dev(self._h, arr, len(items), _t_ptr(results_t)),
                    "relocalize_batch_dev")

    # ---- served form ------------------------------------------------------------------
    def serve_start(self, max_batch: int = 64, max_inflight: int = 2, hbm_budget: int = 0):
        self._check(self._L.relo_serve_start(self._h, max_batch, max_inflight, hbm_budget), "serve_start")

    def submit(self, map_id: int, ranges: np.ndarray, angles: np.ndarray, max_range: float,
               timeout_s: float = 0.0) -> int:
        """Queues a request (relo_submit; relo_submit_until with a deadline of timeout_s seconds)."""
        z = np.ascontiguousarray(ranges, dtype=np.float32)
        a = np.ascontiguousarray(angles, dtype=np.float32)
        t = ctypes.c_int64(0)
        if timeout_s:
            rc = self._L.relo_submit_until(self._h, map_id, _np_ptr(z), _np_ptr(a), len(z), max_range, timeout_s,
                                           ctypes.byref(t))
        else:
            rc = self._L.relo_submit(self._h, map_id, _np_ptr(z), _np_ptr(a), len(z), max_range, ctypes.byref(t))
        self._check(rc, "submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (status, Result, latency seconds)."""
        out = Result()
        lat = ctypes.c_double(0.0)
        rc = self._L.relo_poll(self._h, ticket, ctypes.byref(out), ctypes.byref(lat))
        if rc == PENDING:
            return None
        if rc == E_NOT_FOUND:
            raise ReloError(rc, "unknown ticket")
        return rc, out, lat.value

    def serve_stop(self):
        self._check(self._L.relo_serve_stop(self._h), "serve_stop")

    def stage(self, which: int, dst_t):
        self._check(self._L.relo_get_stage(self._h, which, _t_ptr(dst_t), dst_t.numel() * dst_t.element_size()),
                    "get_stage")
        return dst_t

    def synth_scans(self, map_id: int, cells_t, angles: np.ndarray, max_range: float, ns: int, with_hits=True):
        import torch
        a = np.ascontiguousarray(angles, dtype=np.float32)
        n = cells_t.shape[0]
        r = torch.empty((n, ns), dtype=torch.int32, device=cells_t.device)
        h = torch.empty((n, ns), dtype=torch.int32, device=cells_t.device) if with_hits else None
        ns_out = ctypes.c_int32(0)
        self._check(self._L.relo_synth_scans_dev(self._h, map_id, _t_ptr(cells_t), n, _np_ptr(a), len(a), max_range,
                                                 _t_ptr(r), None if h is None else _t_ptr(h), r.numel(),
                                                 ctypes.byref(ns_out)),
                    "synth_scans")
        if ns_out.value != ns:
            raise ReloError(E_BEAM_GRID, f"N_s is {ns_out.value}, expected {ns}")
        return r, h


def result_from_bytes(b: bytes) -> Result:
    return Result.from_buffer_copy(b)


def tam_class(n_beams: int) -> int:
    """The values-per-lane class of a scan's TAM kernel (relo_tam_class), the key of a TAM tuning entry."""
    return int(lib().relo_tam_class(int(n_beams)))


def probe_l2(stream_bytes: int = 32 << 20, passes: int = 50, gather_log2: int = 24, gathers: int = 1 << 30) -> dict:
    """L2 read rates of this GPU (relo_probe_l2_stream / relo_probe_l2_gather):
    streaming 16-byte loads over an L2-resident buffer, and uniformly random
    2-byte loads from an L2-resident uint16 array.  Returns GB/s and gathers/s."""
    import torch
    L = lib()
    buf = torch.zeros(stream_bytes, dtype=torch.uint8, device="cuda")
    ms = ctypes.c_float(0)
    s = torch.cuda.current_stream().cuda_stream
    rc = L.relo_probe_l2_stream(ctypes.c_void_p(buf.data_ptr()), stream_bytes, passes, ctypes.c_void_p(s),
                                ctypes.byref(ms))
    if rc != OK:
        raise ReloError(rc, "relo_probe_l2_stream")
    stream_gbs = stream_bytes * passes / (ms.value / 1e3) / 1e9
    arr = torch.randint(0, 1 << 15, (1 << gather_log2,), dtype=torch.int16, device="cuda")
    done = ctypes.c_int64(0)
    rc = L.relo_probe_l2_gather(ctypes.c_void_p(arr.data_ptr()), gather_log2, gathers, ctypes.c_void_p(s),
                                ctypes.byref(ms), ctypes.byref(done))
    if rc != OK:
        raise ReloError(rc, "relo_probe_l2_gather")
    gps = done.value / (ms.value / 1e3)
    return {"stream_gbs": stream_gbs, "stream_bytes": stream_bytes,
            "gather_per_s": gps, "gather_2b_gbs": 2.0 * gps / 1e9, "gather_array_bytes": 2 << gather_log2}
