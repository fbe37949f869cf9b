"""CPU oracle for SMAD + TAM relocalization scoring — TEST INFRASTRUCTURE.

A plain, slow FP64 restatement of the paper's scoring path, used only by the
tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The GPU library never imports, links or calls it, and it shares
no code with the GPU library.

Layout: the per-beam / per-pose arithmetic is plain C (``relo_oracle.c``,
built with gcc, no FMA contraction); the sensor plan glue, the ranking and the
batched multi-stage selection are plain Python below.

Paper references (arXiv 2511.01219):
  * Sec. III-A item 3: EDT lookup table            -> edt(), d2_capped()
  * Eq. 11-15: beam grid, FoV intervals, Theta      -> plan()
  * Eq. 13: panoramic synthesized scan              -> synth_scan()
  * Eq. 16-20: SMAD                                 -> smad()
  * Eq. 22-31: TAM and orientation selection        -> tam(), best_orientation()
  * Eq. 21 (Remark 5): CAER in place of SMAD         -> caer()
  * Eq. 32-34: wp_LF, wp_baseline, TAM_mean          -> tam(metric=3, 2, 1)
  * Sec. III overview, Remark 2: ICP refinement of
    the local top-k and re-evaluation               -> icp(), tam_pose(), relocalize(icp_iters=)
  * Sec. III intro, Remarks 2-3, Sec. IV-C params:
    SMAD ordering, batches, local top-k, tau        -> relocalize()

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
except the retention-ratio constants of Eq. 25 and d_max of Eq. 29, whose
values the paper does not print (parity unpinned against the paper for those
two constants; the formulas that use them are pinned).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "relo_oracle.c")
_SO = os.path.join(_HERE, "_relo_oracle.so")
_lib = None

E_BEAM_GRID = -2
E_NO_VALID_BEAMS = -7


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP when available)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "oracle_d2_brute": (I64, [P, I, I, I, I]),
            "oracle_edt_full": (None, [P, I, I, P, I]),
            "oracle_d2_capped": (I64, [P, I, I, I, I, I64]),
            "oracle_beam_grid": (I, [P, I, P, P]),
            "oracle_directions": (None, [I, P]),
            "oracle_intervals": (I, [P, I, I, P, P]),
            "oracle_ranges_q16": (None, [P, I, ctypes.c_float, D, P, P]),
            "oracle_cast_ray": (I64, [P, I, I, I, I, I64, I64, I64, P, P, P]),
            "oracle_synth_scan": (None, [P, I, I, I, I, I, P, I64, P, P, P]),
            "oracle_smad": (None, [P, I, I, P, I, I, P, I64, P, P, I, I64, I, I, P, P, I]),
            "oracle_caer": (None, [P, I, I, P, I, I, P, I64, P, P, I, I, I, P, P, I]),
            "oracle_nearest_occupied": (I, [P, P, I, I, I, I, I64, P, P]),
            "oracle_rigid_fit": (I, [P, P, I, P, P, P]),
            "oracle_icp": (I, [P, P, I, I, D, I64, P, P, I, I, P]),
            "oracle_tam_pose": (None, [P, P, I, I, P, I, P, P, I, P, P, I]),
            "oracle_tam": (None, [P, P, I, I, P, P, I, I, P, P, P, P, I, P, P, P, I]),
            "oracle_max_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data


def max_threads() -> int:
    return int(_L().oracle_max_threads())


# ----------------------------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------------------------

@dataclass
class Params:
    """Constants of Eq. 23-31 and of the batched inference.

    z_hit, sigma_hit, z_rand: Sec. IV-B (Case 1); eps: Eq. 23; batch 200,
    local top-20, tau 0.95: Sec. IV-C.  The four retention-ratio endpoints of
    Eq. 25 and d_max of Eq. 29 are not printed in the paper; the values here
    make alpha fall as the FoV grows, as the text after Eq. 25 describes.
    """
    z_hit: float = 1.0
    sigma_hit: float = 0.2
    z_rand: float = 0.0
    eps: float = 1e-6
    d_max: float = 2.0
    a_mid_min: float = 0.9
    a_mid_max: float = 0.8
    a_low_min: float = 0.8
    a_low_max: float = 0.6
    panoramic_ratio: float = 0.9
    n_orient: int = 360
    topk: int = 256
    batch: int = 200
    local_topk: int = 20
    tau: float = 0.95
    n_skip_beam: int = 1
    coarse: int = 0     # ranking metric: 0 SMAD (Eq. 16-20), 1 CAER (Eq. 21), 3 none (Table II, no ordering)
    fine: int = 0       # scoring metric: 0 TAM (Eq. 31), 1 TAM_mean (Eq. 34), 2 wp_baseline (Eq. 33), 3 wp_LF (Eq. 32)


# ----------------------------------------------------------------------------------------------
# EDT
# ----------------------------------------------------------------------------------------------

def edt(grid: np.ndarray, n_threads: int = 0) -> np.ndarray:
    """Squared EDT in cells (int64, -1 if the map has no occupied cell)."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    out = np.empty((H, W), np.int64)
    _L().oracle_edt_full(_p(g), W, H, _p(out), n_threads or max_threads())
    return out


def d2_brute(grid: np.ndarray, x: int, y: int) -> int:
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    return int(_L().oracle_d2_brute(_p(g), W, H, x, y))


def d2_capped(grid: np.ndarray, x: int, y: int, cap: int) -> int:
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    return int(_L().oracle_d2_capped(_p(g), W, H, x, y, cap))


# ----------------------------------------------------------------------------------------------
# sensor plan (Eq. 11-16)
# ----------------------------------------------------------------------------------------------

class PlanError(ValueError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


def plan(ranges, angles, max_range: float, res: float, prm: Params) -> dict:
    """Everything about one scan that does not depend on a hypothesis."""
    z = np.ascontiguousarray(np.asarray(ranges, np.float32)[:: prm.n_skip_beam])        # Eq. 11
    a = np.ascontiguousarray(np.asarray(angles, np.float32)[:: prm.n_skip_beam])
    n = int(z.size)
    L = _L()
    b = np.zeros(n, np.int32)
    ns = ctypes.c_int32(0)
    rc = L.oracle_beam_grid(_p(a), n, ctypes.byref(ns), _p(b))
    if rc != 0:
        raise PlanError(rc, "beam angles are not on a uniform panoramic grid")
    ns = int(ns.value)
    n_orient = prm.n_orient if prm.n_orient > 0 else ns
    if ns % n_orient != 0:
        raise PlanError(E_BEAM_GRID, "n_orient must divide N_s")
    n_enum = ns // n_orient                                                                  # Eq. 15
    D = np.zeros(2 * ns, np.int64)
    L.oracle_directions(ns, _p(D))
    u = np.zeros(n, np.int32)
    ln = np.zeros(n, np.int32)
    K = int(L.oracle_intervals(_p(b), n, ns, _p(u), _p(ln)))                               # Eq. 12
    R = np.zeros(n, np.int64)
    valid = np.zeros(n, np.uint8)
    L.oracle_ranges_q16(_p(z), n, ctypes.c_float(max_range), res, _p(R), _p(valid))
    lam = float(ln[:K].sum()) / ns                                                          # lambda
    a_mid = prm.a_mid_min + lam * (prm.a_mid_max - prm.a_mid_min)                          # Eq. 25
    a_low = prm.a_low_min + lam * (prm.a_low_max - prm.a_low_min)
    return dict(n=n, ns=ns, b=b, D=D, u=u[:K].copy(), len=ln[:K].copy(), K=K, R=R, valid=valid,
                n_valid=int(valid.sum()), sum_real=int(R.sum()), lam=lam, n_orient=n_orient, n_enum=n_enum,
                panoramic=lam >= prm.panoramic_ratio, a_mid=a_mid, a_low=a_low,
                rmax_q16=rmax_q16(max_range, res), res=res, max_range=max_range)


def rmax_q16(max_range: float, res: float) -> int:
    """llrint(max_range * 65536 / res), max_range taken as float32."""
    v = float(np.float32(max_range)) * 65536.0 / res
    return int(np.rint(v))


# ----------------------------------------------------------------------------------------------
# synthesized scan, SMAD
# ----------------------------------------------------------------------------------------------

def cast_ray(grid, hx, hy, Dx, Dy, rmax_q16_):
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    hx_, hy_, st = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    r = _L().oracle_cast_ray(_p(g), W, H, hx, hy, Dx, Dy, rmax_q16_, ctypes.byref(hx_), ctypes.byref(hy_),
                             ctypes.byref(st))
    return int(r), (int(hx_.value), int(hy_.value)), int(st.value)


def synth_scan(grid, hx: int, hy: int, pl: dict):
    """Eq. 13: the N_s synthesized Q16 ranges from one hypothesis and the hit cells (-1 if none)."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    ns = pl["ns"]
    r = np.zeros(ns, np.int64)
    hxs = np.zeros(ns, np.int32)
    hys = np.zeros(ns, np.int32)
    _L().oracle_synth_scan(_p(g), W, H, hx, hy, ns, _p(pl["D"]), pl["rmax_q16"], _p(r), _p(hxs), _p(hys))
    return r, hxs, hys


def smad(grid, hyps: np.ndarray, pl: dict, n_threads: int = 0):
    """Eq. 16-20 for every hypothesis: (numerator int64, minimising m int32)."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    h = np.ascontiguousarray(hyps, dtype=np.int32)
    n = len(h)
    num = np.zeros(n, np.int64)
    mm = np.zeros(n, np.int32)
    _L().oracle_smad(_p(g), W, H, _p(h), n, pl["ns"], _p(pl["D"]), pl["rmax_q16"], _p(pl["u"]), _p(pl["len"]),
                     pl["K"], pl["sum_real"], pl["n_enum"], int(pl["panoramic"]), _p(num), _p(mm),
                     n_threads or max_threads())
    return num, mm


def smad_metres(num, pl: dict) -> np.ndarray:
    """SMAD value of Eq. 19 in metres from the Q16 numerator."""
    return np.asarray(num, np.float64) / float(pl["len"].sum()) / 65536.0 * pl["res"]


def caer(grid, hyps: np.ndarray, pl: dict, n_threads: int = 0):
    """Eq. 21 for every hypothesis: (numerator int64, minimising m int32), the
    numerator being the sum over the FoV beams of |R_i - synthesized range|
    (Q16; invalid beams count 0), minimised over the orientations SMAD uses."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    h = np.ascontiguousarray(hyps, dtype=np.int32)
    n = len(h)
    num = np.zeros(n, np.int64)
    mm = np.zeros(n, np.int32)
    R = np.ascontiguousarray(pl["R"], dtype=np.int64)
    _L().oracle_caer(_p(g), W, H, _p(h), n, pl["ns"], _p(pl["D"]), pl["rmax_q16"], _p(pl["b"]), _p(R), pl["n"],
                     pl["n_enum"], int(pl["panoramic"]), _p(num), _p(mm), n_threads or max_threads())
    return num, mm


def coarse(grid, hyps: np.ndarray, pl: dict, prm: "Params", n_threads: int = 0):
    """The ranking metric prm.coarse selects: SMAD (0), CAER (1), or none (3:
    the Table II arm without SMAD ordering, where TAM takes the hypotheses in
    their own order: every numerator 0 at m = 0, so rank() keeps the index
    order)."""
    if prm.coarse == 3:
        return np.zeros(len(hyps), np.int64), np.zeros(len(hyps), np.int32)
    return caer(grid, hyps, pl, n_threads) if prm.coarse == 1 else smad(grid, hyps, pl, n_threads)


def rank(num: np.ndarray, k: int) -> np.ndarray:
    """SMAD ordering: hypotheses sorted by (numerator, index), first k kept."""
    order = sorted(range(len(num)), key=lambda i: (int(num[i]), i))
    return np.asarray(order[:k], np.int64)


# ----------------------------------------------------------------------------------------------
# TAM
# ----------------------------------------------------------------------------------------------

def tam(grid, pairs_xy: np.ndarray, pairs_m: np.ndarray, pl: dict, prm: Params, res: float,
        d2tab: np.ndarray | None = None, n_threads: int = 0, components: bool = False, metric: int | None = None):
    """Eq. 23-31 for each (hypothesis cell, m) pair; float64 scores.  metric
    (default prm.fine): 0 TAM, 1 TAM_mean (Eq. 34), 2 wp_baseline (Eq. 33),
    3 wp_LF (Eq. 32)."""
    if pl["n_valid"] == 0:
        raise PlanError(E_NO_VALID_BEAMS, "scan has no valid beam")
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    xy = np.ascontiguousarray(pairs_xy, dtype=np.int32)
    mm = np.ascontiguousarray(pairs_m, dtype=np.int32)
    n = len(mm)
    out = np.zeros(n, np.float64)
    comp = np.zeros((n, 5), np.float64) if components else None
    params = np.array([prm.z_hit, prm.sigma_hit, prm.z_rand, prm.eps, res, prm.d_max, pl["a_mid"], pl["a_low"],
                       float(prm.fine if metric is None else metric)], np.float64)
    d2c = None if d2tab is None else np.ascontiguousarray(d2tab, dtype=np.int64)
    d2p = None if d2c is None else _p(d2c)
    _L().oracle_tam(_p(g), d2p, W, H, _p(xy), _p(mm), n, pl["ns"], _p(pl["D"]), _p(pl["b"]), _p(pl["R"]),
                    _p(pl["valid"]), pl["n"], _p(params), _p(out), None if comp is None else _p(comp),
                    n_threads or max_threads())
    return (out, comp) if components else out


def tam_grid(grid, hyps: np.ndarray, sel: np.ndarray, pl: dict, prm: Params, res: float, d2tab=None,
             n_threads: int = 0) -> np.ndarray:
    """TAM for every selected hypothesis and every m in Theta: [len(sel), n_orient]."""
    m_list = np.arange(pl["n_orient"], dtype=np.int32) * pl["n_enum"]
    xy = np.repeat(np.asarray(hyps, np.int32)[sel], len(m_list), axis=0)
    mm = np.tile(m_list, len(sel))
    T = tam(grid, xy, mm, pl, prm, res, d2tab, n_threads)
    return T.reshape(len(sel), len(m_list))


# ----------------------------------------------------------------------------------------------
# ICP refinement and re-evaluation at continuous poses
# ----------------------------------------------------------------------------------------------

def scan_points(pl: dict, res: float):
    """The valid beams as sensor-frame ranges (metres) and angles: z_i =
    R_i res / 65536 (the Q16 range) and a_i = 2 pi b_i / N_s (its panoramic
    grid angle), so a continuous pose (cell centre, theta_m) reproduces the
    endpoints of the integer rule up to rounding."""
    v = pl["valid"].astype(bool)
    z = np.ascontiguousarray(pl["R"][v].astype(np.float64) * res / 65536.0)
    a = np.ascontiguousarray(pl["b"][v].astype(np.float64) * (2.0 * math.pi / pl["ns"]))
    return z, a


def _clamp(prm: Params, res: float) -> int:
    return int(round(prm.d_max / res)) ** 2


def nearest_occupied(grid, x: int, y: int, cap: int, d2tab=None):
    """The nearest occupied cell to cell (x, y) within squared cell distance
    cap (ties: smaller dy, then smaller dx), or None."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    d2c = None if d2tab is None else np.ascontiguousarray(d2tab, dtype=np.int64)
    ox, oy = ctypes.c_int(0), ctypes.c_int(0)
    ok = _L().oracle_nearest_occupied(_p(g), None if d2c is None else _p(d2c), W, H, x, y, cap, ctypes.byref(ox),
                                      ctypes.byref(oy))
    return (int(ox.value), int(oy.value)) if ok else None


def rigid_fit(w: np.ndarray, c: np.ndarray):
    """(phi, tx, ty) minimising sum |R(phi) w_i + t - c_i|^2, or None for fewer than 2 pairs."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    phi, tx, ty = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    ok = _L().oracle_rigid_fit(_p(w), _p(c), len(w), ctypes.byref(phi), ctypes.byref(tx), ctypes.byref(ty))
    return (phi.value, tx.value, ty.value) if ok else None


def icp_points(grid, pose, z, a, res: float, C: int, iters: int, d2tab=None):
    """ICP of the beams (z, a) from pose (x, y, theta): (refined pose, iterations)."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    d2c = None if d2tab is None else np.ascontiguousarray(d2tab, dtype=np.int64)
    ps = np.array(pose, np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    it = _L().oracle_icp(_p(g), None if d2c is None else _p(d2c), W, H, res, C, _p(z), _p(a), len(z), iters, _p(ps))
    return ps, int(it)


def icp(grid, pose, pl: dict, prm: Params, res: float, iters: int, d2tab=None):
    """ICP of the scan's valid beams from pose, pairs kept within d_max."""
    z, a = scan_points(pl, res)
    return icp_points(grid, pose, z, a, res, _clamp(prm, res), iters, d2tab)


def tam_pose(grid, poses, pl: dict, prm: Params, res: float, d2tab=None, metric: int | None = None,
             n_threads: int = 0) -> np.ndarray:
    """The score (prm.fine unless metric is given) at continuous poses [n, 3] for the scan's valid beams."""
    g = np.ascontiguousarray(grid, dtype=np.int8)
    H, W = g.shape
    ps = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 3))
    z, a = scan_points(pl, res)
    params = np.array([prm.z_hit, prm.sigma_hit, prm.z_rand, prm.eps, res, prm.d_max, pl["a_mid"], pl["a_low"],
                       float(prm.fine if metric is None else metric)], np.float64)
    d2c = None if d2tab is None else np.ascontiguousarray(d2tab, dtype=np.int64)
    out = np.zeros(len(ps), np.float64)
    _L().oracle_tam_pose(_p(g), None if d2c is None else _p(d2c), W, H, _p(ps), len(ps), _p(z), _p(a), len(z),
                         _p(params), _p(out), n_threads or max_threads())
    return out


def best_orientation(T_row) -> int:
    """Eq. 22: argmax over Theta, ties to the smaller m (returns the position in Theta)."""
    best = 0
    for q in range(1, len(T_row)):
        if T_row[q] > T_row[best]:
            best = q
    return best


# ----------------------------------------------------------------------------------------------
# the whole path
# ----------------------------------------------------------------------------------------------

def relocalize(grid, res: float, hyps: np.ndarray, ranges, angles, max_range: float, prm: Params,
               d2tab: np.ndarray | None = None, n_threads: int = 0, early_stop: bool = True,
               icp_iters: int = 0) -> dict:
    """SMAD ranking (CAER with prm.coarse = 1), then batched TAM orientation
    selection (the metric prm.fine picks) with local top-k and early
    termination (Sec. III intro).  With icp_iters > 0 each local top-k pose
    is refined by icp_iters ICP iterations and scored again at its continuous
    pose (tam_pose); a batch's best is then the best re-evaluated score, and
    the result is that refined pose.  With icp_iters = 0 the re-evaluated
    score of a local top-k pose is its first TAM score.

    With early_stop False every survivor is scored (the "TAM on the top K"
    form); otherwise batches stop after the first whose best score >= tau.
    """
    pl = plan(ranges, angles, max_range, res, prm)
    if len(hyps) == 0:
        raise ValueError("no hypotheses")
    num, m_smad = coarse(grid, hyps, pl, prm, n_threads)
    K = min(prm.topk, len(hyps))
    surv = rank(num, K)
    if d2tab is None and grid.size <= (1 << 21):
        d2tab = edt(grid, n_threads)
    B = min(prm.batch, K)
    best = None
    batches = []
    n_tam = 0
    per_hyp = {}
    for start in range(0, K, B):
        members = surv[start:start + B]
        T = tam_grid(grid, hyps, members, pl, prm, res, d2tab, n_threads)
        n_tam += T.size
        scored = []
        for r, h in enumerate(members):
            q = best_orientation(T[r])
            per_hyp[int(h)] = (q * pl["n_enum"], float(T[r, q]))
            scored.append((float(T[r, q]), start + r, int(h), q * pl["n_enum"]))
        scored.sort(key=lambda t: (-t[0], t[1]))
        local = scored[: prm.local_topk]
        batches.append(local)
        reev = []
        for (t0, pos, h, m) in local:   # re-evaluation of the local top-k, in local order
            pose = ((hyps[h][0] + 0.5) * res, (hyps[h][1] + 0.5) * res, m * 2.0 * math.pi / pl["ns"])
            if icp_iters > 0:
                pose, _ = icp(grid, pose, pl, prm, res, icp_iters, d2tab)
                t0 = float(tam_pose(grid, [pose], pl, prm, res, d2tab)[0])
            reev.append((t0, pos, h, m, tuple(float(v) for v in pose)))
        top = max(reev, key=lambda t: (t[0], -t[1]))
        if best is None or top[0] > best[0]:
            best = top
        if early_stop and top[0] >= prm.tau:
            break
    T_best, rank_pos, h, m, pose = best
    theta = math.remainder(pose[2], 2.0 * math.pi)
    if theta >= math.pi:
        theta -= 2.0 * math.pi
    return dict(hyp=h, m=m, tam=T_best, x=pose[0], y=pose[1], theta=theta,
                smad_num=int(num[h]), smad=float(smad_metres(num[h], pl)), survivors=surv, smad_nums=num,
                smad_m=m_smad, per_hyp=per_hyp, batches=batches, n_batches=len(batches),
                n_smad_evals=0 if prm.coarse == 3 else len(hyps) * (1 if pl["panoramic"] else pl["n_orient"]),
                n_tam_evals=n_tam,
                plan=pl)
