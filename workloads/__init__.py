"""Seeded synthetic workloads for passive 2-D global relocalization.

Everything here is *input generation*: occupancy grids shaped like the paper's
indoor scenes (Sec. IV-A: 0.05 m grids of rooms, corridors and repetitive
layouts), LiDAR scans produced by a continuous-geometry sensor simulator, and
positional hypotheses from a traversability-constrained RRT (Algorithm 1).
None of the scoring arithmetic (EDT, synthesized scans, SMAD, TAM) lives here;
both the CPU oracle and the GPU library consume these arrays.

Conventions shared by every generator:
  * grids are int8, row-major (row = y), values 0 free / 100 occupied / -1
    unknown; the map origin is (0, 0) and cell (cx, cy) covers
    [cx*res, (cx+1)*res) x [cy*res, (cy+1)*res);
  * scan angles lie on a uniform panoramic grid of N_s directions
    (2*pi*j/N_s), stored as float32 in [-pi, pi), increasing across the FoV;
  * hypotheses are returned both as integer cells and as cell-centre
    coordinates in metres.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_RRT_SRC = os.path.join(_HERE, "rrt.c")
_RRT_SO = os.path.join(_HERE, "_rrt.so")
_lib = None

FREE, OCC, UNKNOWN = 0, 100, -1


def build(force: bool = False) -> str:
    """Compile the RRT sampler (plain C, host only)."""
    if force or not os.path.exists(_RRT_SO) or os.path.getmtime(_RRT_SO) < os.path.getmtime(_RRT_SRC):
        tmp = _RRT_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", _RRT_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _RRT_SO)
    return _RRT_SO


def _rrt_lib():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_RRT_SO)
        lib.wl_rrt_sample.restype = ctypes.c_int
        lib.wl_rrt_sample.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        _lib = lib
    return _lib


# ----------------------------------------------------------------------------------------------
# maps
# ----------------------------------------------------------------------------------------------

def make_room(seed: int, n: int = 64, n_boxes: int = 6, box_min: int = 2, box_max: int = 8) -> np.ndarray:
    """n x n room with 1-cell walls and axis-aligned box obstacles of box_min..box_max cells."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, n), np.int8)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = OCC
    for _ in range(n_boxes):
        w, h = rng.integers(box_min, box_max + 1, size=2)
        x0 = int(rng.integers(2, n - 2 - w))
        y0 = int(rng.integers(2, n - 2 - h))
        g[y0:y0 + h, x0:x0 + w] = OCC
    return g


def make_office(seed: int, n: int = 1024, res: float = 0.05, corridor_m: float = 1.5, min_room_m: float = 4.0,
                max_room_m: float = 9.0, door_m: float = 0.9, unknown_frac: float = 0.03) -> np.ndarray:
    """BSP office: rooms with 1-cell walls and doors, separated by corridors.

    The outside of the building is unknown (-1): a border band sized so that
    about ``unknown_frac`` of all cells are unknown.  A few furniture blocks
    are dropped into rooms.
    """
    rng = np.random.default_rng(seed)
    band = max(1, int(round(unknown_frac * n / 4.0)))
    g = np.full((n, n), UNKNOWN, np.int8)
    lo, hi = band, n - band          # building interior is [lo, hi)
    g[lo:hi, lo:hi] = FREE
    g[lo, lo:hi] = g[hi - 1, lo:hi] = OCC
    g[lo:hi, lo] = g[lo:hi, hi - 1] = OCC
    cor = max(2, int(round(corridor_m / res)))
    min_room = int(round(min_room_m / res))
    max_room = int(round(max_room_m / res))
    door = max(2, int(round(door_m / res)))
    rooms = []

    def wall_with_door(axis: int, pos: int, a: int, b: int):
        """Wall along `axis` (0: horizontal at row pos, 1: vertical at col pos) over [a, b) with one door."""
        if axis == 0:
            g[pos, a:b] = OCC
        else:
            g[a:b, pos] = OCC
        if b - a > door + 4:
            d0 = int(rng.integers(a + 2, b - door - 2))
            if axis == 0:
                g[pos, d0:d0 + door] = FREE
            else:
                g[d0:d0 + door, pos] = FREE

    def split(x0, y0, x1, y1, depth):
        w, h = x1 - x0, y1 - y0
        big = max(w, h)
        if big <= max_room or (big < 2 * min_room + cor):
            rooms.append((x0, y0, x1, y1))
            return
        if w >= h:
            s = int(rng.integers(x0 + min_room, x1 - min_room - cor + 1))
            # corridor occupies columns [s, s+cor); walls at s-1 and s+cor bound the two halves
            wall_with_door(1, s, y0, y1)
            wall_with_door(1, s + cor - 1, y0, y1)
            split(x0, y0, s, y1, depth + 1)
            split(s + cor, y0, x1, y1, depth + 1)
        else:
            s = int(rng.integers(y0 + min_room, y1 - min_room - cor + 1))
            wall_with_door(0, s, x0, x1)
            wall_with_door(0, s + cor - 1, x0, x1)
            split(x0, y0, x1, s, depth + 1)
            split(x0, s + cor, x1, y1, depth + 1)

    split(lo + 1, lo + 1, hi - 1, hi - 1, 0)
    # interior partitions inside large leaf rooms and some furniture
    for (x0, y0, x1, y1) in rooms:
        w, h = x1 - x0, y1 - y0
        if w > 2 * min_room // 2 + 20 and rng.random() < 0.5:
            s = int(rng.integers(x0 + w // 3, x1 - w // 3))
            wall_with_door(1, s, y0, y1)
        for _ in range(int(rng.integers(0, 4))):
            bw, bh = (int(v) for v in rng.integers(8, 30, size=2))
            if w - bw - 8 <= 4 or h - bh - 8 <= 4:
                continue
            bx = int(rng.integers(x0 + 4, x1 - bw - 4))
            by = int(rng.integers(y0 + 4, y1 - bh - 4))
            g[by:by + bh, bx:bx + bw] = OCC
    return g


def make_warehouse(seed: int, n: int = 4096, res: float = 0.05, shelf_m: float = 1.0, aisle_m: float = 3.0,
                   shelf_len_m: float | None = None, cross_m: float = 2.5, margin_m: float = 4.0) -> np.ndarray:
    """Warehouse with perimeter walls and periodic, identical shelving rows.

    Shelf rows run along x, ``shelf_m`` deep, separated by ``aisle_m`` aisles,
    and are cut every ``shelf_len_m`` by ``cross_m`` cross aisles; the layout
    repeats exactly, so many positions see near-identical scans.
    """
    rng = np.random.default_rng(seed)
    g = np.zeros((n, n), np.int8)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = OCC
    if shelf_len_m is None:   # 20 m runs, shorter on small maps so at least two fit across
        shelf_len_m = min(20.0, (n * res - 2 * margin_m - cross_m) / 2.0)
    sh = int(round(shelf_m / res))
    ai = int(round(aisle_m / res))
    sl = int(round(shelf_len_m / res))
    cr = int(round(cross_m / res))
    mg = int(round(margin_m / res))
    y = mg
    while y + sh < n - mg:
        x = mg
        while x + sl <= n - mg:
            g[y:y + sh, x:x + sl] = OCC
            x += sl + cr
        y += sh + ai
    # a handful of pillars along the margins break the perfect symmetry only slightly
    for _ in range(8):
        px = int(rng.integers(4, n - 8))
        py = int(rng.choice([int(rng.integers(4, max(5, mg - 8))), int(rng.integers(n - mg + 4, n - 8))]))
        g[py:py + 6, px:px + 6] = OCC
    return g


# ----------------------------------------------------------------------------------------------
# sensor geometry and scans
# ----------------------------------------------------------------------------------------------

def choose_ns(n_beams: int, fov_deg: float, n_orient: int) -> int:
    """Panoramic beam count N_s for a sensor with n_beams over about fov_deg.

    N_s is a multiple of n_orient (so the orientation set of Eq. 15 has a
    whole stride) and n_beams <= N_s <= 2 n_beams (FoV between 180 and 360 deg).
    """
    q = int(round(n_beams * 360.0 / (fov_deg * n_orient)))
    q_lo = -(-n_beams // n_orient)
    q_hi = (2 * n_beams) // n_orient
    q = min(max(q, q_lo), max(q_lo, q_hi))
    return n_orient * q


def beam_angles(n_beams: int, n_s: int) -> np.ndarray:
    """float32 angles of n_beams consecutive panoramic directions centred on 0 (sensor forward)."""
    b0 = -(n_beams // 2)
    j = np.arange(b0, b0 + n_beams, dtype=np.float64)
    a = j * (2.0 * math.pi / n_s)
    a = (a + math.pi) % (2.0 * math.pi) - math.pi
    return a.astype(np.float32)


def render_scan(grid: np.ndarray, res: float, pose, angles: np.ndarray, max_range: float) -> np.ndarray:
    """Noise-free LiDAR ranges from a continuous pose.

    Each beam is a ray from (x, y) at world angle theta + angle; its range is
    the distance at which it enters the first occupied cell (value >= 65),
    measured exactly against the cell squares.  Unknown cells do not stop a
    beam.  Beams that leave the map or travel max_range return max_range.
    """
    H, W = grid.shape
    x0, y0, th = (float(v) for v in pose)
    ang = th + angles.astype(np.float64)
    dx, dy = np.cos(ang), np.sin(ang)
    px, py = x0 / res, y0 / res                      # position in cell units
    cx = np.full(ang.shape, int(math.floor(px)), np.int64)
    cy = np.full(ang.shape, int(math.floor(py)), np.int64)
    sx = np.where(dx > 0, 1, -1)
    sy = np.where(dy > 0, 1, -1)
    with np.errstate(divide="ignore"):
        tdx = np.where(dx != 0, 1.0 / np.abs(dx), np.inf)
        tdy = np.where(dy != 0, 1.0 / np.abs(dy), np.inf)
    fx, fy = px - math.floor(px), py - math.floor(py)
    tx = np.where(dx > 0, (1.0 - fx) * tdx, np.where(dx < 0, fx * tdx, np.inf))
    ty = np.where(dy > 0, (1.0 - fy) * tdy, np.where(dy < 0, fy * tdy, np.inf))
    limit = max_range / res
    out = np.full(ang.shape, max_range, np.float64)
    alive = np.ones(ang.shape, bool)
    occ = grid >= 65
    while alive.any():
        stepx = alive & (tx <= ty)
        stepy = alive & ~(tx <= ty)
        t = np.where(stepx, tx, ty)
        cx = np.where(stepx, cx + sx, cx)
        cy = np.where(stepy, cy + sy, cy)
        tx = np.where(stepx, tx + tdx, tx)
        ty = np.where(stepy, ty + tdy, ty)
        far = alive & (t >= limit)
        off = alive & ((cx < 0) | (cy < 0) | (cx >= W) | (cy >= H))
        alive &= ~(far | off)
        hit = np.zeros_like(alive)
        idx = np.nonzero(alive)[0]
        if idx.size:
            hit[idx] = occ[cy[idx], cx[idx]]
        out = np.where(hit, t * res, out)
        alive &= ~hit
    return out.astype(np.float32)


def add_noise(z: np.ndarray, max_range: float, seed: int, sigma: float = 0.02, drop_frac: float = 0.05,
              short_frac: float = 0.10, short_min: float = 0.1) -> np.ndarray:
    """Noise model of the office workload: short returns from unmapped
    obstacles (10 %, uniform in [0.1 m, z]), Gaussian range noise sigma, and
    5 % of beams dropped to max range (no return)."""
    rng = np.random.default_rng(seed)
    z = z.astype(np.float64).copy()
    n = z.size
    ret = z < max_range
    short = rng.random(n) < short_frac
    sel = short & ret & (z > short_min)
    z[sel] = rng.uniform(short_min, z[sel])
    z[ret] += rng.normal(0.0, sigma, size=int(ret.sum()))
    z = np.clip(z, 1e-3, max_range)
    z[rng.random(n) < drop_frac] = max_range
    return z.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# hypotheses
# ----------------------------------------------------------------------------------------------

def clearance_table(grid: np.ndarray, res: float) -> np.ndarray:
    """Per-cell clearance (metres) for the RRT: distance from each cell centre to
    the nearest occupied or unknown cell centre (map outside counts as blocked),
    from SciPy's exact Euclidean distance transform."""
    from scipy.ndimage import distance_transform_edt
    open_ = np.pad(grid == FREE, 1, constant_values=False)
    return (distance_transform_edt(open_)[1:-1, 1:-1] * res).astype(np.float32)


def free_start(grid: np.ndarray, res: float, r_robot: float, seed: int, clr: np.ndarray | None = None):
    """A seeded free cell centre (metres) with clearance >= 2 r_robot if one exists, else >= r_robot."""
    clr = clearance_table(grid, res) if clr is None else clr
    rng = np.random.default_rng(seed)
    for need in (2 * r_robot, r_robot):
        ok = np.argwhere(clr >= need)
        if len(ok):
            cy, cx = ok[int(rng.integers(len(ok)))]
            return (cx + 0.5) * res, (cy + 0.5) * res
    raise RuntimeError("no free start point with the requested clearance")


def rrt(grid: np.ndarray, res: float, p0, rho: float, eta_max: float = 0.6, r_robot: float = 0.21,
        eps_gain: int = 2, seed: int = 0, max_rounds: int = 200, cap: int = 4_000_000,
        clr: np.ndarray | None = None):
    """Run Algorithm 1; returns (xy [n,2] float64 metres, n_nodes, n_rounds)."""
    lib = _rrt_lib()
    H, W = grid.shape
    clr = np.ascontiguousarray(clearance_table(grid, res) if clr is None else clr, dtype=np.float32)
    out = np.zeros((cap, 2), np.float64)
    nn, nr = ctypes.c_int(0), ctypes.c_int(0)
    n = lib.wl_rrt_sample(clr.ctypes.data, W, H, res, float(p0[0]), float(p0[1]), rho, eta_max, r_robot,
                          eps_gain, seed, max_rounds, out.ctypes.data, cap, ctypes.byref(nn), ctypes.byref(nr))
    if n < 0:
        raise RuntimeError("RRT sampler failed")
    return out[:n].copy(), nn.value, nr.value


def rrt_hypotheses(grid: np.ndarray, res: float, n_hyp: int, seed: int, r_robot: float = 0.21,
                   eta_max: float = 0.6, eps_gain: int = 2):
    """Exactly n_hyp RRT hypotheses: rho is shrunk until Algorithm 1 yields at
    least n_hyp voxel representatives, then a seeded subset is kept.  Returns
    integer cells [n, 2] (cx, cy) int32, sorted by cell index."""
    H, W = grid.shape
    clr = clearance_table(grid, res)
    p0 = free_start(grid, res, r_robot, seed, clr)
    free_area = float((clr >= r_robot).sum()) * res * res
    rho = math.sqrt(free_area / (1.1 * n_hyp))
    for _ in range(30):
        xy, _, _ = rrt(grid, res, p0, rho, eta_max, r_robot, eps_gain, seed, clr=clr)
        if len(xy) >= n_hyp:
            break
        rho *= 0.85
    else:
        raise RuntimeError("RRT could not produce enough hypotheses")
    rng = np.random.default_rng(seed + 17)
    pick = np.sort(rng.choice(len(xy), size=n_hyp, replace=False))
    cells = np.floor(xy[pick] / res).astype(np.int64)
    cells = np.unique(cells, axis=0)
    while len(cells) < n_hyp:          # two picks in one cell: top up from the rest
        extra = np.floor(xy / res).astype(np.int64)
        cells = np.unique(np.concatenate([cells, extra]), axis=0)[: n_hyp]
    cells = cells[:n_hyp]
    order = np.lexsort((cells[:, 0], cells[:, 1]))
    return cells[order].astype(np.int32), rho


def free_hypotheses(grid: np.ndarray, res: float, n_hyp: int, seed: int, r_robot: float = 0.21,
                    clr: np.ndarray | None = None) -> np.ndarray:
    """n_hyp distinct seeded cells whose clearance is at least r_robot (int32 [n, 2], sorted).

    A fast stand-in for Algorithm 1 where many large maps must be generated
    (the batched and served workloads): uniform over the traversable cells
    instead of the RRT's voxel representatives."""
    clr = clearance_table(grid, res) if clr is None else clr
    ok = np.argwhere(clr >= r_robot)[:, ::-1]
    rng = np.random.default_rng(seed)
    pick = ok[rng.choice(len(ok), size=min(n_hyp, len(ok)), replace=False)]
    order = np.lexsort((pick[:, 0], pick[:, 1]))
    return pick[order].astype(np.int32)


def scan_for(grid: np.ndarray, res: float, hyps: np.ndarray, n_beams: int, n_s: int, n_orient: int,
             max_range: float, seed: int, noisy: bool = True):
    """(angles, ranges, ground-truth pose) of a seeded scan near a random hypothesis."""
    return _scan_for(grid, res, hyps, n_beams, n_s, n_orient, max_range, seed, noisy)


@dataclass
class Instance:
    grid: np.ndarray
    res: float
    hyps: np.ndarray
    ranges: np.ndarray
    angles: np.ndarray
    max_range: float
    topk: int
    n_s: int


BEAM_COUNTS = (541, 720, 1081, 1440)


def batched_instances(seed: int = 1003, count: int = 64, n_orient: int = 360):
    """The batched workload: `count` independent relocalizations.

    Map sides uniform over {512, 576, ..., 2048} cells (office for even draws,
    warehouse for odd), beam counts from {541, 720, 1081, 1440} with a FoV
    drawn in [180, 360] deg (N_s a multiple of n_orient in [N, 2N]), 1k-20k
    hypotheses, TAM on the top 256 (maps up to 1024^2) or 1024, 25 m range,
    office noise model."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.integers(8, 33)) * 64
        s_i = seed * 100 + i
        grid = make_office(s_i, n=side) if i % 2 == 0 else make_warehouse(s_i, n=side)
        n_beams = int(rng.choice(BEAM_COUNTS))
        fov = float(rng.uniform(180.0, 360.0))
        n_s = choose_ns(n_beams, fov, n_orient)
        n_hyp = int(rng.integers(1000, 20001))
        hyps = free_hypotheses(grid, 0.05, n_hyp, s_i)
        angles, z, _ = _scan_for(grid, 0.05, hyps, n_beams, n_s, n_orient, 25.0, s_i, True)
        out.append(Instance(grid, 0.05, hyps, z, angles, 25.0, 256 if side <= 1024 else 1024, n_s))
    return out


def served_maps(seed: int = 1004):
    """The served workload's 8 resident maps: two each of 512^2, 1024^2, 2048^2
    and 4096^2 (one office, one warehouse) with 1250 / 5000 / 10000 / 20000
    hypotheses."""
    out = []
    for k, (side, n_hyp) in enumerate(((512, 1250), (1024, 5000), (2048, 10000), (4096, 20000))):
        for j in range(2):
            s_i = seed * 100 + 2 * k + j
            grid = make_office(s_i, n=side) if j == 0 else make_warehouse(s_i, n=side)
            out.append((grid, 0.05, free_hypotheses(grid, 0.05, n_hyp, s_i)))
    return out


def served_scans(maps, per_map: int = 6, seed: int = 1004, n_orient: int = 360):
    """A pool of seeded scans per resident map (beam counts as the batched workload)."""
    rng = np.random.default_rng(seed + 1)
    pool = []
    for mi, (grid, res, hyps) in enumerate(maps):
        for j in range(per_map):
            n_beams = int(rng.choice(BEAM_COUNTS))
            n_s = choose_ns(n_beams, float(rng.uniform(180.0, 360.0)), n_orient)
            angles, z, _ = _scan_for(grid, res, hyps, n_beams, n_s, n_orient, 25.0, seed * 1000 + mi * 10 + j, True)
            pool.append((mi, z, angles, 25.0))
    return pool


def sweep_poses(wl, n_pos: int = 15, step_m: float = 0.1, n_orient_sweep: int = 36, orient_step_deg: int = 10):
    """The poses of a translation-affinity sweep in the manner of Fig. 8: n_pos
    cells step_m apart through the scan's true position along the first axis
    (x, then y) whose cells are all free, and n_orient_sweep orientations
    orient_step_deg apart starting at the true one (on a grid of 360
    orientations).  Returns (cells int32 [n_pos, 2], offsets in cells, axis
    name, orientation indices q of the 360-grid)."""
    gx, gy, gth = wl.gt_pose
    cx, cy = int(round(gx / wl.res - 0.5)), int(round(gy / wl.res - 0.5))
    step = int(round(step_m / wl.res))
    offs = (np.arange(n_pos) - n_pos // 2) * step
    free = wl.grid < 65
    for ax, (dx, dy) in enumerate(((1, 0), (0, 1))):
        cells = np.stack([cx + dx * offs, cy + dy * offs], 1)
        inside = ((cells[:, 0] >= 0) & (cells[:, 0] < wl.grid.shape[1]) & (cells[:, 1] >= 0) &
                  (cells[:, 1] < wl.grid.shape[0]))
        if inside.all() and free[cells[:, 1], cells[:, 0]].all():
            m_true = int(round(gth / (2 * math.pi) * wl.n_s)) % wl.n_s
            q_true = m_true // (wl.n_s // 360)
            qs = [(q_true + orient_step_deg * j) % 360 for j in range(n_orient_sweep)]
            return cells.astype(np.int32), offs, "xy"[ax], qs
    raise RuntimeError("no axis through the true position with all sweep cells free")


def cell_centres(cells: np.ndarray, res: float) -> np.ndarray:
    return (cells.astype(np.float64) + 0.5) * res


# ----------------------------------------------------------------------------------------------
# full workloads
# ----------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: np.ndarray
    res: float
    hyps: np.ndarray            # int32 [N_h, 2] cells (cx, cy)
    ranges: np.ndarray          # float32 [N]
    angles: np.ndarray          # float32 [N]
    max_range: float
    n_orient: int
    topk: int
    n_s: int
    gt_pose: tuple
    extra: dict = field(default_factory=dict)


def _scan_for(grid, res, hyps, n_beams, n_s, n_orient, max_range, seed, noisy):
    rng = np.random.default_rng(seed + 5)
    angles = beam_angles(n_beams, n_s)
    h = hyps[int(rng.integers(len(hyps)))]
    # ground truth: near a hypothesis (within half a cell-size jitter of 0.3 m) on free space
    for _ in range(1000):
        x = (h[0] + 0.5) * res + rng.uniform(-0.3, 0.3)
        y = (h[1] + 0.5) * res + rng.uniform(-0.3, 0.3)
        cx, cy = int(math.floor(x / res)), int(math.floor(y / res))
        if 0 <= cx < grid.shape[1] and 0 <= cy < grid.shape[0] and grid[cy, cx] == FREE:
            break
    else:
        x, y = (h[0] + 0.5) * res, (h[1] + 0.5) * res
    m = int(rng.integers(n_orient)) * (n_s // n_orient)
    th = m * 2.0 * math.pi / n_s
    th = (th + math.pi) % (2 * math.pi) - math.pi
    z = render_scan(grid, res, (x, y, th), angles, max_range)
    if noisy:
        z = add_noise(z, max_range, seed + 9)
    return angles, z, (x, y, th)


def config(i: int, seed: int | None = None) -> Workload:
    """The seeded synthetic workloads (seed = 1000 + i unless given).

    0: 64x64 room, 360 beams (N_s = 504, ~257 deg), 72 orientations, 200
       hypotheses, top 16, noise-free.
    1: 1024x1024 office, 1081 beams (N_s = 1440, ~270 deg), 360 orientations,
       5000 hypotheses, top 256, noise model of add_noise().
    2: 4096x4096 warehouse, 1440 beams over 360 deg, 720 orientations, 20000
       hypotheses, top 1024, same noise model.

    With the environment variable RELO_WORKLOAD_CACHE naming a directory, a
    generated workload is saved there and read back by later calls (input
    generation only; the arrays are the same).
    """
    seed = 1000 + i if seed is None else seed
    cache = os.environ.get("RELO_WORKLOAD_CACHE")
    path = os.path.join(cache, f"config{i}_{seed}.npz") if cache else None
    if path and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return Workload(name=f"config{i}", grid=z["grid"], res=float(z["res"]), hyps=z["hyps"], ranges=z["ranges"],
                        angles=z["angles"], max_range=float(z["max_range"]), n_orient=int(z["n_orient"]),
                        topk=int(z["topk"]), n_s=int(z["n_s"]), gt_pose=tuple(float(v) for v in z["gt"]),
                        extra={"rho": float(z["rho"]), "seed": seed})
    wl = _config(i, seed)
    if path:
        os.makedirs(cache, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, grid=wl.grid, res=wl.res, hyps=wl.hyps, ranges=wl.ranges, angles=wl.angles,
                 max_range=wl.max_range, n_orient=wl.n_orient, topk=wl.topk, n_s=wl.n_s, gt=np.array(wl.gt_pose),
                 rho=wl.extra["rho"])
        os.replace(tmp, path)
    return wl


def _config(i: int, seed: int) -> Workload:
    res = 0.05
    if i == 0:
        grid = make_room(seed)
        hyps, rho = rrt_hypotheses(grid, res, 200, seed)
        n_beams, n_orient, max_range, topk, noisy = 360, 72, 10.0, 16, False
        n_s = choose_ns(n_beams, 270.0, n_orient)
    elif i == 1:
        grid = make_office(seed)
        hyps, rho = rrt_hypotheses(grid, res, 5000, seed)
        n_beams, n_orient, max_range, topk, noisy = 1081, 360, 25.0, 256, True
        n_s = choose_ns(n_beams, 270.0, n_orient)
    elif i == 2:
        grid = make_warehouse(seed)
        hyps, rho = rrt_hypotheses(grid, res, 20000, seed)
        n_beams, n_orient, max_range, topk, noisy = 1440, 720, 25.0, 1024, True
        n_s = 1440
    else:
        raise ValueError("config must be 0, 1 or 2")
    angles, z, gt = _scan_for(grid, res, hyps, n_beams, n_s, n_orient, max_range, seed, noisy)
    return Workload(name=f"config{i}", grid=grid, res=res, hyps=hyps, ranges=z, angles=angles,
                    max_range=max_range, n_orient=n_orient, topk=topk, n_s=n_s, gt_pose=gt,
                    extra={"rho": rho, "seed": seed})
