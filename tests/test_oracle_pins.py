"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to brute force on tiny inputs, to exact
rational geometry, to a closed form, or to an invariant of the paper's
definitions, chosen so that a dropped term, a wrong sign, an off-by-one index
or a transposed operand fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

RES = 0.05


def rand_grid(rng, H, W, p):
    g = np.where(rng.random((H, W)) < p, 100, 0).astype(np.int8)
    g[rng.random((H, W)) < 0.05] = -1
    return g


# ------------------------------------------------------------------------------------------
# EDT (Sec. III-A item 3)
# ------------------------------------------------------------------------------------------

def brute_d2(grid):
    occ = np.argwhere(grid >= 65)
    H, W = grid.shape
    out = np.full((H, W), -1, np.int64)
    if len(occ) == 0:
        return out
    yy, xx = np.mgrid[0:H, 0:W]
    d = (yy[..., None] - occ[:, 0]) ** 2 + (xx[..., None] - occ[:, 1]) ** 2
    return d.min(axis=-1).astype(np.int64)


@pytest.mark.parametrize("seed", range(6))
def test_edt_full_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 24)), int(rng.integers(1, 24))
    g = rand_grid(rng, H, W, [0.0, 0.02, 0.1, 0.5, 1.0, 0.01][seed])
    assert np.array_equal(oracle.edt(g), brute_d2(g))


def test_edt_single_obstacle_is_squared_distance():
    g = np.zeros((9, 13), np.int8)
    g[2, 7] = 100
    d = oracle.edt(g)
    assert d[2, 7] == 0 and d[0, 0] == 4 + 49 and d[8, 12] == 36 + 25


@pytest.mark.parametrize("seed", range(4))
def test_d2_capped_and_brute(seed):
    rng = np.random.default_rng(100 + seed)
    g = rand_grid(rng, 20, 17, 0.04)
    ref = brute_d2(g)
    for _ in range(60):
        x, y = int(rng.integers(17)), int(rng.integers(20))
        cap = int(rng.integers(1, 80))
        want = cap if ref[y, x] < 0 else min(int(ref[y, x]), cap)
        assert oracle.d2_capped(g, x, y, cap) == want
        assert oracle.d2_brute(g, x, y) == ref[y, x]


# ------------------------------------------------------------------------------------------
# integer ray casting (Eq. 13)
# ------------------------------------------------------------------------------------------

def exact_traversal(grid, hx, hy, Dx, Dy, rmax_q16):
    """Cells whose squares the ray from the centre of (hx, hy) crosses with
    positive length, ordered by entry parameter (slab clipping, exact
    rationals); stops as the method does.  Returns (hit_cell or None, n_cells,
    tie_seen)."""
    H, W = grid.shape
    px, py = Fraction(2 * hx + 1, 2), Fraction(2 * hy + 1, 2)
    cells = []
    n = max(H, W) + 2
    for cy in range(-1, H + 1):
        for cx in range(-1, W + 1):
            lo, hi = Fraction(0), Fraction(10 ** 9)
            ok = True
            for p, d, c in ((px, Dx, cx), (py, Dy, cy)):
                if d == 0:
                    if not (c < p < c + 1):
                        ok = False
                else:
                    t1, t2 = Fraction(c - p) / d, Fraction(c + 1 - p) / d
                    if t1 > t2:
                        t1, t2 = t2, t1
                    lo, hi = max(lo, t1), min(hi, t2)
            if ok and hi > lo and hi > 0 and (cx, cy) != (hx, hy):
                cells.append((lo, cx, cy))
    cells.sort()
    ties = any(cells[i][0] == cells[i + 1][0] for i in range(len(cells) - 1))
    cnt = 0
    for _, cx, cy in cells:
        cnt += 1
        if cx < 0 or cy < 0 or cx >= W or cy >= H:
            return None, cnt, ties
        c2 = (cx - hx) ** 2 + (cy - hy) ** 2
        if c2 * (1 << 32) > rmax_q16 * rmax_q16:
            return None, cnt, ties
        if grid[cy, cx] >= 65:
            return (cx, cy), cnt, ties
    return None, cnt, ties


@pytest.mark.parametrize("seed", range(5))
def test_cast_ray_matches_exact_geometry(seed):
    rng = np.random.default_rng(200 + seed)
    g = rand_grid(rng, 14, 16, 0.12)
    g[7, 8] = 0
    checked = 0
    for _ in range(80):
        ang = rng.uniform(-math.pi, math.pi)
        Dx, Dy = int(round(math.cos(ang) * 2 ** 30)), int(round(math.sin(ang) * 2 ** 30))
        rmax = int(rng.integers(2, 12)) * 65536 + int(rng.integers(65536))
        want_hit, want_n, ties = exact_traversal(g, 8, 7, Dx, Dy, rmax)
        if ties:
            continue
        r, hit, steps = oracle.cast_ray(g, 8, 7, Dx, Dy, rmax)
        assert steps == want_n
        if want_hit is None:
            assert r == 0 and hit == (-1, -1)
        else:
            assert hit == want_hit
            c2 = (hit[0] - 8) ** 2 + (hit[1] - 7) ** 2
            assert r == math.isqrt(c2 << 32)
        checked += 1
    assert checked > 60


def test_cast_ray_axis_and_corner_tie():
    g = np.zeros((9, 9), np.int8)
    g[4, 8] = 100
    r, hit, steps = oracle.cast_ray(g, 4, 4, 1 << 30, 0, 100 * 65536)
    assert hit == (8, 4) and r == 4 * 65536 and steps == 4
    # 45 degrees: the ray passes exactly through cell corners; x is stepped first
    g = np.zeros((9, 9), np.int8)
    g[5, 5] = 100                      # reached as (4,4)->(5,4)->(5,5)
    g[5, 4] = 100                      # would be hit first if y were stepped first
    r, hit, steps = oracle.cast_ray(g, 4, 4, 759250125, 759250125, 100 * 65536)
    assert hit == (5, 5) and steps == 2 and r == math.isqrt(2 << 32)


def test_cast_ray_range_limit_and_off_map():
    g = np.zeros((5, 40), np.int8)
    g[2, 30] = 100
    assert oracle.cast_ray(g, 2, 2, 1 << 30, 0, 28 * 65536 - 1)[0] == 0      # centre beyond range
    assert oracle.cast_ray(g, 2, 2, 1 << 30, 0, 28 * 65536)[0] == 28 * 65536  # exactly at range: hit
    assert oracle.cast_ray(g, 2, 2, -(1 << 30), 0, 100 * 65536)[1] == (-1, -1)  # leaves map


# ------------------------------------------------------------------------------------------
# beam grid, intervals, directions (Eq. 11-15)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,ns", [(360, 504), (1081, 1440), (1440, 1440), (541, 1080), (2, 8)])
def test_beam_grid_recovers_ns(n, ns):
    a = workloads.beam_angles(n, ns)
    pl = oracle.plan(np.ones(n, np.float32), a, 10.0, RES, oracle.Params(n_orient=0))
    assert pl["ns"] == ns
    b0 = -(n // 2)
    assert list(pl["b"]) == [(b0 + i) % ns for i in range(n)]
    assert pl["K"] == 1 and pl["len"][0] == n and pl["u"][0] == (b0 % ns if n < ns else 0)
    assert pl["lam"] == n / ns


def test_beam_grid_rejects_off_grid_and_duplicates():
    a = workloads.beam_angles(100, 400).astype(np.float64)
    a[37] += 0.01 * 2 * math.pi / 400
    with pytest.raises(oracle.PlanError):
        oracle.plan(np.ones(100, np.float32), a.astype(np.float32), 10.0, RES, oracle.Params(n_orient=0))
    a = workloads.beam_angles(100, 400)
    a[5] = a[4]
    with pytest.raises(oracle.PlanError):
        oracle.plan(np.ones(100, np.float32), a, 10.0, RES, oracle.Params(n_orient=0))


def test_intervals_with_gap_and_wrap():
    ns = 360
    b = [i % ns for i in list(range(350, 370)) + list(range(100, 110))]
    L = oracle._L()
    bb = np.array(sorted(b), np.int32)
    u = np.zeros(30, np.int32)
    ln = np.zeros(30, np.int32)
    K = L.oracle_intervals(bb.ctypes.data, len(bb), ns, u.ctypes.data, ln.ctypes.data)
    got = sorted(zip(u[:K].tolist(), ln[:K].tolist()))
    assert got == [(100, 10), (350, 20)]


def test_directions():
    D = np.zeros(2 * 8, np.int64)
    oracle._L().oracle_directions(8, D.ctypes.data)
    D = D.reshape(8, 2)
    s = round(2 ** 30 / math.sqrt(2))
    assert D.tolist() == [[2 ** 30, 0], [s, s], [0, 2 ** 30], [-s, s], [-2 ** 30, 0], [-s, -s], [0, -2 ** 30],
                          [s, -s]]


def test_ranges_q16_and_validity():
    z = np.array([1.0, 0.0, -1.0, np.nan, np.inf, 9.99, 10.0, 0.025], np.float32)
    pl = oracle.plan(z, workloads.beam_angles(8, 16), 10.0, RES, oracle.Params(n_orient=0))
    assert pl["valid"].tolist() == [1, 0, 0, 0, 0, 1, 0, 1]
    assert pl["R"][0] == 20 * 65536 and pl["R"][7] == 32768
    assert pl["R"][5] == int(np.rint(float(np.float32(9.99)) * 65536.0 / RES))
    assert pl["sum_real"] == int(pl["R"].sum())


# ------------------------------------------------------------------------------------------
# SMAD (Eq. 16-20)
# ------------------------------------------------------------------------------------------

def room_case(seed, n_beams=90, ns=120, n_orient=40):
    g = workloads.make_room(seed, n=40, n_boxes=4)
    hyps = np.argwhere(g == 0)[:, ::-1]
    rng = np.random.default_rng(seed)
    hyps = hyps[rng.choice(len(hyps), 25, replace=False)].astype(np.int32)
    return g, hyps, workloads.beam_angles(n_beams, ns), n_orient


def self_rendered(g, h, m, pl, angles):
    """Real scan equal to the oracle's synthesized scan at (h, m): beam i reads
    synthesized beam (b_i + m) mod N_s, converted back to metres."""
    syn, _, _ = oracle.synth_scan(g, int(h[0]), int(h[1]), pl)
    j = (pl["b"] + m) % pl["ns"]
    return (syn[j].astype(np.float64) * RES / 65536.0).astype(np.float32)


@pytest.mark.parametrize("seed", range(3))
def test_smad_direct_equals_prefix_sum_form(seed):
    g, hyps, ang, n_orient = room_case(seed)
    prm = oracle.Params(n_orient=n_orient)
    z = np.random.default_rng(seed).uniform(0.1, 3.0, len(ang)).astype(np.float32)
    z[::7] = 0.0
    pl = oracle.plan(z, ang, 4.0, RES, prm)
    num, mm = oracle.smad(g, hyps, pl)
    ns = pl["ns"]
    for h in range(len(hyps)):
        syn, _, _ = oracle.synth_scan(g, int(hyps[h, 0]), int(hyps[h, 1]), pl)
        S = np.concatenate([[0], np.cumsum(np.concatenate([syn, syn]))])     # Eq. 17, S[0] = 0
        best = None
        for m in range(0, ns, pl["n_enum"]):
            # Eq. 18, 0-based; the window start is reduced mod N_s so it stays on the 2 N_s extension
            W = sum(int(S[(u + m) % ns + L] - S[(u + m) % ns]) for u, L in zip(pl["u"], pl["len"]))
            v = abs(pl["sum_real"] - W)
            if best is None or v < best[0]:
                best = (v, m)
        assert (num[h], mm[h]) == best


@pytest.mark.parametrize("seed", range(3))
def test_smad_zero_at_self_rendered_pose(seed):
    g, hyps, ang, n_orient = room_case(seed)
    prm = oracle.Params(n_orient=n_orient)
    pl0 = oracle.plan(np.ones(len(ang), np.float32), ang, 6.0, RES, prm)
    h, m = hyps[3], 7 * pl0["n_enum"]
    z = self_rendered(g, h, m, pl0, ang)
    pl = oracle.plan(z, ang, 6.0, RES, prm)
    num, mm = oracle.smad(g, hyps, pl)
    assert num[3] == 0
    assert oracle.rank(num, 1)[0] in np.nonzero(num == 0)[0]


def test_smad_panoramic_uses_m0_only():
    g, hyps, _, _ = room_case(1)
    ang = workloads.beam_angles(120, 120)
    z = np.random.default_rng(0).uniform(0.2, 2.0, 120).astype(np.float32)
    pl = oracle.plan(z, ang, 6.0, RES, oracle.Params(n_orient=40))
    assert pl["lam"] == 1.0 and pl["panoramic"]
    num, mm = oracle.smad(g, hyps, pl)
    assert (mm == 0).all()
    for h in range(5):   # with a full circle every rotation has the same window sum
        syn, _, _ = oracle.synth_scan(g, int(hyps[h, 0]), int(hyps[h, 1]), pl)
        assert num[h] == abs(pl["sum_real"] - int(syn.sum()))


def test_rank_ties_by_index():
    num = np.array([5, 3, 5, 3, 1, 3], np.int64)
    assert oracle.rank(num, 6).tolist() == [4, 1, 3, 5, 0, 2]
    assert oracle.best_orientation([0.2, 0.5, 0.5, 0.1]) == 1


# ------------------------------------------------------------------------------------------
# TAM (Eq. 22-31): closed forms
# ------------------------------------------------------------------------------------------

def ell(d, p):
    return math.log(p.z_hit * math.exp(-d * d / (2 * p.sigma_hit ** 2)) + p.z_rand + p.eps)


def test_tam_all_endpoints_on_obstacles():
    g = np.full((30, 30), 100, np.int8)
    g[15, 15] = 0
    prm = oracle.Params(n_orient=8)
    ang = workloads.beam_angles(50, 64)
    z = np.full(50, 4 * RES, np.float32)
    pl = oracle.plan(z, ang, 10.0, RES, prm)
    T, comp = oracle.tam(g, np.array([[15, 15]] * 8), np.arange(8) * 8, pl, prm, RES, components=True)
    want = (1.0 + 1e-6) ** (1.0 / 3.0)
    assert np.allclose(T, want, rtol=0, atol=1e-15)
    assert np.allclose(comp[:, 2], 1.0) and np.allclose(comp[:, 3], 1.0)


def _endpoints_on_row(hy, row, D, b, rng, ns):
    """ranges (metres, float32) for which each beam's endpoint lands on `row`."""
    z = []
    for bi in b:
        Dy = int(D[2 * (bi % ns) + 1])
        t = (row - hy) / (Dy / 2 ** 30)          # cells along the beam
        z.append(t * RES)
    return np.array(z, np.float32)


def test_tam_equal_distances_closed_form():
    H, W = 200, 200
    g = np.zeros((H, W), np.int8)
    g[150, :] = 100                       # a wall along a row
    ns, n = 64, 9
    ang = workloads.beam_angles(n, ns)    # beams within +-0.44 rad of +y after a quarter turn
    prm = oracle.Params(n_orient=16)
    pl0 = oracle.plan(np.ones(n, np.float32), ang, 100.0, RES, prm)
    m = ns // 4                           # sensor forward = +y
    b = (pl0["b"] + m) % ns
    hx, hy, row = 100, 100, 147           # endpoints on row 147: 3 cells from the wall
    z = _endpoints_on_row(hy, row, pl0["D"], b, None, ns)
    pl = oracle.plan(z, ang, 100.0, RES, prm)
    # confirm the endpoint rule sends every beam to row 147
    for i in range(n):
        j = (pl["b"][i] + m) % ns
        oy = (int(pl["R"][i]) * int(pl["D"][2 * j + 1]) + (1 << 45)) >> 46
        assert hy + oy == row
    T, comp = oracle.tam(g, np.array([[hx, hy]]), np.array([m]), pl, prm, RES, components=True)
    d = 3 * RES
    wp = math.exp(ell(d, prm))
    sd = 1 - (d - RES / 2) / (prm.d_max - RES / 2)
    assert math.isclose(T[0], (wp * sd * 1.0) ** (1 / 3), rel_tol=1e-12)
    assert math.isclose(comp[0, 3], 1.0, rel_tol=1e-12)


def test_tam_two_distance_classes_closed_form():
    """n1 beams on the wall (d = 0) and n2 beams off the map (d = d_max):
    retention (Eq. 25-27), the median, s_d (Eq. 29) and the population
    variance (Eq. 30) all follow in closed form."""
    H, W = 120, 120
    g = np.zeros((H, W), np.int8)
    g[60:, :] = 100                       # lower half solid
    ns, n = 200, 100
    ang = workloads.beam_angles(n, ns)
    prm = oracle.Params(n_orient=20)
    m = 0                                 # forward = +x: the beams with sin > 0.3 point into the solid half
    hx, hy = 60, 59
    pl0 = oracle.plan(np.ones(n, np.float32), ang, 1000.0, RES, prm)
    z = np.empty(n, np.float32)
    n1 = 0
    for i in range(n):
        j = (pl0["b"][i] + m) % ns
        Dx, Dy = pl0["D"][2 * j] / 2 ** 30, pl0["D"][2 * j + 1] / 2 ** 30
        if Dy > 0.3:        # points into the solid lower half (y grows)
            z[i] = 10 * RES; n1 += 1
        else:               # leaves the map
            z[i] = 500 * RES
    pl = oracle.plan(z, ang, 1000.0, RES, prm)
    T, comp = oracle.tam(g, np.array([[hx, hy]]), np.array([m]), pl, prm, RES, components=True)
    N, n2 = n, n - n1
    lam = n / ns
    a_mid = prm.a_mid_min + lam * (prm.a_mid_max - prm.a_mid_min)
    k_mid = max(1, math.floor(a_mid * N))
    l0, l1 = ell(0.0, prm), ell(prm.d_max, prm)
    top_mean = (min(k_mid, n1) * l0 + max(0, k_mid - n1) * l1) / k_mid
    p = n2 / N
    dbar = p * prm.d_max
    var = p * (1 - p) * prm.d_max ** 2
    sd = 1 - (max(dbar, RES / 2) - RES / 2) / (prm.d_max - RES / 2)
    want = (math.exp(top_mean) * sd * math.exp(-var / 2)) ** (1 / 3)
    assert 0 < n1 < N
    assert math.isclose(comp[0, 0], top_mean, rel_tol=1e-12)
    assert math.isclose(T[0], want, rel_tol=1e-12)


def test_tam_median_is_kmid_mean_and_sd_can_vanish():
    """The running mean of a descending list never increases, so the median of
    Eq. 27 is the k_mid mean; a pose whose mean distance reaches d_max gets
    s_d = 0 and T = 0."""
    g = np.zeros((100, 100), np.int8)
    g[0, 0] = 100
    prm = oracle.Params(n_orient=4)
    ang = workloads.beam_angles(40, 64)
    pl = oracle.plan(np.full(40, 0.5, np.float32), ang, 10.0, RES, prm)
    T = oracle.tam(g, np.array([[60, 60]]), np.array([0]), pl, prm, RES)
    assert T[0] == 0.0
    rng = np.random.default_rng(3)
    for _ in range(200):
        v = np.sort(rng.uniform(-14, 0, rng.integers(1, 50)))[::-1]
        means = np.cumsum(v) / np.arange(1, len(v) + 1)
        assert np.all(np.diff(means) <= 1e-12)


# ------------------------------------------------------------------------------------------
# Eq. 21 and Eq. 32-34: the metrics the paper sets against SMAD and TAM
# ------------------------------------------------------------------------------------------

def two_class_case():
    """The scene of test_tam_two_distance_classes_closed_form: n1 beams end on
    the solid half (d = 0), the others leave the map (d = d_max)."""
    H, W = 120, 120
    g = np.zeros((H, W), np.int8)
    g[60:, :] = 100
    ns, n = 200, 100
    ang = workloads.beam_angles(n, ns)
    prm = oracle.Params(n_orient=20)
    pl0 = oracle.plan(np.ones(n, np.float32), ang, 1000.0, RES, prm)
    z = np.empty(n, np.float32)
    n1 = 0
    for i in range(n):
        j = pl0["b"][i] % ns
        if pl0["D"][2 * j + 1] / 2 ** 30 > 0.3:
            z[i] = 10 * RES
            n1 += 1
        else:
            z[i] = 500 * RES
    return g, prm, oracle.plan(z, ang, 1000.0, RES, prm), n1, n


def test_fine_metrics_two_distance_classes_closed_form():
    """wp_LF sums l over every beam, n1 l(0) + n2 l(d_max), with no retention
    (Eq. 32); wp_baseline is (exp(wp_LF / N) s_d)^(1/2) (Eq. 33); TAM_mean is
    the arithmetic mean of the retained exp(L_bar), s_d and c (Eq. 34)."""
    g, prm, pl, n1, N = two_class_case()
    n2 = N - n1
    l0, l1 = ell(0.0, prm), ell(prm.d_max, prm)
    lam = N / pl["ns"]
    k_mid = max(1, math.floor((prm.a_mid_min + lam * (prm.a_mid_max - prm.a_mid_min)) * N))
    wp = math.exp((min(k_mid, n1) * l0 + max(0, k_mid - n1) * l1) / k_mid)
    p = n2 / N
    sd = 1 - (max(p * prm.d_max, RES / 2) - RES / 2) / (prm.d_max - RES / 2)
    c = math.exp(-p * (1 - p) * prm.d_max ** 2 / 2)
    lf = n1 * l0 + n2 * l1
    xy, m = np.array([[60, 59]]), np.array([0])
    got = [oracle.tam(g, xy, m, pl, prm, RES, metric=k)[0] for k in range(4)]
    assert math.isclose(got[0], (wp * sd * c) ** (1 / 3), rel_tol=1e-12)
    assert math.isclose(got[1], (wp + sd + c) / 3, rel_tol=1e-12)
    assert math.isclose(got[2], math.sqrt(math.exp(lf / N) * sd), rel_tol=1e-12)
    assert math.isclose(got[3], lf, rel_tol=1e-12)
    assert 0 < n1 < N and got[2] < got[0]   # the unretained off-map beams pull the baseline down


def test_fine_metrics_all_endpoints_on_obstacles():
    """d = 0 for every beam: l = log(z_hit + z_rand + eps) = log wp, s_d = c = 1."""
    g = np.full((30, 30), 100, np.int8)
    g[15, 15] = 0
    prm = oracle.Params(n_orient=8)
    ang = workloads.beam_angles(50, 64)
    pl = oracle.plan(np.full(50, 4 * RES, np.float32), ang, 10.0, RES, prm)
    wp = 1.0 + 1e-6
    xy, m = np.array([[15, 15]] * 8), np.arange(8) * 8
    for k, want in ((1, (wp + 2) / 3), (2, math.sqrt(wp)), (3, 50 * math.log(wp))):
        assert np.allclose(oracle.tam(g, xy, m, pl, prm, RES, metric=k), want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("seed", range(3))
def test_fine_metric_bounds(seed):
    """Arithmetic mean >= geometric mean of (wp, s_d, c): TAM_mean >= TAM;
    every l <= log(z_hit + z_rand + eps), so wp_LF <= N log(...) and
    wp_baseline <= 1."""
    g, hyps, ang, n_orient = room_case(seed)
    prm = oracle.Params(n_orient=n_orient)
    z = np.random.default_rng(seed).uniform(0.1, 3.0, len(ang)).astype(np.float32)
    pl = oracle.plan(z, ang, 4.0, RES, prm)
    xy = np.repeat(hyps[:8], 5, axis=0)
    m = np.tile(np.arange(5) * 3 * pl["n_enum"], 8)
    T, comp = oracle.tam(g, xy, m, pl, prm, RES, components=True, metric=0)
    Tm = oracle.tam(g, xy, m, pl, prm, RES, metric=1)
    Tb = oracle.tam(g, xy, m, pl, prm, RES, metric=2)
    Tl = oracle.tam(g, xy, m, pl, prm, RES, metric=3)
    assert np.all(Tm >= T * (1 - 1e-14)) and np.any(Tm > T * (1 + 1e-3))
    assert np.all((Tb >= 0) & (Tb <= 1))
    assert np.all(Tl <= pl["n_valid"] * math.log(prm.z_hit + prm.z_rand + prm.eps) + 1e-9)
    assert np.allclose((Tm * 3 - comp[:, 2] - comp[:, 3]), comp[:, 1], rtol=1e-12)   # same components as TAM


@pytest.mark.parametrize("seed", range(3))
def test_caer_bounds_smad(seed):
    """|sum (a - b)| <= sum |a - b| at every m, so the minimum CAER numerator
    is at least the minimum SMAD numerator (Eq. 19 vs Eq. 21)."""
    g, hyps, ang, n_orient = room_case(seed)
    prm = oracle.Params(n_orient=n_orient)
    z = np.random.default_rng(seed).uniform(0.1, 3.0, len(ang)).astype(np.float32)
    z[::9] = 0.0
    pl = oracle.plan(z, ang, 4.0, RES, prm)
    cn, cm = oracle.caer(g, hyps, pl)
    sn, sm = oracle.smad(g, hyps, pl)
    assert np.all(cn >= sn) and np.any(cn > sn)
    assert np.all(cm % pl["n_enum"] == 0)


def test_caer_equals_smad_when_every_real_range_is_longer():
    """Real ranges all longer than every synthesized range (a 40-cell room,
    real beams at 3.9 m): every beam difference is positive, the triangle
    inequality is an equality, and CAER and SMAD agree in value and m."""
    g, hyps, ang, n_orient = room_case(2)
    prm = oracle.Params(n_orient=n_orient)
    pl = oracle.plan(np.full(len(ang), 3.9, np.float32), ang, 4.0, RES, prm)
    cn, cm = oracle.caer(g, hyps, pl)
    sn, sm = oracle.smad(g, hyps, pl)
    assert np.array_equal(cn, sn) and np.array_equal(cm, sm)


def test_caer_on_a_map_without_obstacles():
    """No obstacle: every synthesized range is 0 (no hit), so the numerator is
    the sum of the real Q16 ranges at every m and the first m is kept."""
    g = np.zeros((50, 50), np.int8)
    ang = workloads.beam_angles(90, 120)
    z = np.random.default_rng(5).uniform(0.1, 2.0, 90).astype(np.float32)
    z[::11] = np.inf
    pl = oracle.plan(z, ang, 3.0, RES, oracle.Params(n_orient=40))
    hyps = np.array([[5, 5], [25, 30], [49, 0]], np.int32)
    cn, cm = oracle.caer(g, hyps, pl)
    want = sum(int(np.rint(float(v) * 65536.0 / RES)) for v in z if np.isfinite(v) and 0 < v < 3.0)
    assert cn.tolist() == [want] * 3 and cm.tolist() == [0] * 3


# ------------------------------------------------------------------------------------------
# ICP refinement and re-evaluation at continuous poses (Sec. III overview, Remark 2)
# ------------------------------------------------------------------------------------------

def test_rigid_fit_recovers_a_rigid_motion():
    """Pairs related exactly by a rotation and a translation give them back."""
    rng = np.random.default_rng(0)
    for phi, t in ((0.3, (1.5, -0.7)), (-2.9, (0.0, 4.0)), (1e-7, (1e-7, 0.0))):
        w = rng.uniform(-5, 5, (12, 2))
        R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
        c = w @ R.T + np.array(t)
        f, tx, ty = oracle.rigid_fit(w, c)
        assert math.isclose(f, phi, abs_tol=1e-12) and np.allclose((tx, ty), t, atol=1e-12)
    assert oracle.rigid_fit(np.zeros((1, 2)), np.zeros((1, 2))) is None


def test_nearest_occupied_ties_and_range():
    """Four occupied cells at squared distance 25 from (20, 20) ((+-3, +-4)
    and (0, 5)): the first in (dy, dx) order is (17, 16); beyond cap: none."""
    g = np.zeros((41, 41), np.int8)
    for dx, dy in ((3, 4), (-3, 4), (0, 5), (3, -4)):
        g[20 + dy, 20 + dx] = 100
    d2 = oracle.edt(g)
    assert d2[20, 20] == 25
    assert oracle.nearest_occupied(g, 20, 20, 25, d2) == (23, 16)   # dy = -4 first, then dx = +3
    assert oracle.nearest_occupied(g, 20, 20, 24, d2) is None
    assert oracle.nearest_occupied(g, 20, 20, 25) == (23, 16)       # without the table: the capped search


def pillar_scene():
    """Occupied single cells far apart (>= 6 cells), and beams aimed exactly
    at their centres from a true pose."""
    g = np.zeros((120, 120), np.int8)
    pillars = [(20, 30), (90, 25), (100, 80), (35, 95), (60, 60), (15, 70), (75, 105), (105, 45)]
    for x, y in pillars:
        g[y, x] = 100
    true = (55.3 * RES, 48.7 * RES, 0.4)
    z, a = [], []
    for x, y in pillars:
        cx, cy = (x + 0.5) * RES, (y + 0.5) * RES
        z.append(math.hypot(cx - true[0], cy - true[1]))
        a.append(math.atan2(cy - true[1], cx - true[0]) - true[2])
    return g, true, np.array(z), np.array(a)


def test_icp_one_step_on_exact_pairs():
    """From a pose off by 0.6 cm, -0.7 cm and 0.1 degree every beam still falls
    next to its own pillar, the pairs are exact, and one fit lands on the
    true pose; the next iteration moves nothing."""
    g, true, z, a = pillar_scene()
    C = int(round(2.0 / RES)) ** 2
    start = (true[0] + 0.006, true[1] - 0.007, true[2] + math.radians(0.1))
    pose, it = oracle.icp_points(g, start, z, a, RES, C, 1)
    assert it == 1 and np.allclose(pose, true, atol=1e-10)
    pose2, it2 = oracle.icp_points(g, start, z, a, RES, C, 10)
    assert it2 == 2 and np.allclose(pose2, true, atol=1e-10)


def test_icp_drops_pairs_beyond_d_max():
    """Beams that end in open space with no occupied cell within d_max (here 4
    cells, C = 16) take no part: the result is the same with or without them."""
    g, true, z, a = pillar_scene()
    C = 16
    start = (true[0] + 0.006, true[1] - 0.007, true[2] + math.radians(0.1))
    za = np.concatenate([z, [0.3, 0.45]])               # endpoints 6 and 9 cells from the pose, far from every pillar
    aa = np.concatenate([a, [2.0, -2.5]])
    for i in (len(z), len(z) + 1):
        wx = start[0] + za[i] * math.cos(start[2] + aa[i])
        wy = start[1] + za[i] * math.sin(start[2] + aa[i])
        assert oracle.nearest_occupied(g, int(wx // RES), int(wy // RES), C) is None
        assert oracle.nearest_occupied(g, int(wx // RES), int(wy // RES), 40 ** 2) is not None
    p1, _ = oracle.icp_points(g, start, z, a, RES, C, 5)
    p2, _ = oracle.icp_points(g, start, za, aa, RES, C, 5)
    assert np.array_equal(p1, p2)


def test_tam_at_continuous_pose_equals_integer_rule_away_from_cell_edges():
    """At a hypothesis cell centre and orientation theta_m the continuous
    endpoint floor((x_c + z cos) / res) equals the integer rule cell +
    round-half-up(R D / 2^46) unless the endpoint lies within 1e-6 cells of a
    cell edge; wherever no beam does, the two scores are equal."""
    g, hyps, ang, n_orient = room_case(1)
    prm = oracle.Params(n_orient=n_orient)
    z = np.random.default_rng(1).uniform(0.1, 1.5, len(ang)).astype(np.float32)
    pl = oracle.plan(z, ang, 4.0, RES, prm)
    zz, aa = oracle.scan_points(pl, RES)
    d2 = oracle.edt(g)
    checked = 0
    for h in hyps[:10]:
        for m in range(0, pl["ns"], 7 * pl["n_enum"]):
            pose = ((h[0] + 0.5) * RES, (h[1] + 0.5) * RES, m * 2 * math.pi / pl["ns"])
            ex = (pose[0] + zz * np.cos(pose[2] + aa)) / RES
            ey = (pose[1] + zz * np.sin(pose[2] + aa)) / RES
            margin = min(np.abs(ex - np.round(ex)).min(), np.abs(ey - np.round(ey)).min())
            if margin < 1e-6:
                continue
            t_int = oracle.tam(g, np.array([h]), np.array([m]), pl, prm, RES, d2)[0]
            t_pose = oracle.tam_pose(g, [pose], pl, prm, RES, d2)[0]
            assert t_int == t_pose
            checked += 1
    assert checked >= 20


def test_relocalize_with_icp_refines_a_noise_free_pose():
    """A scan rendered from a pose between cells: with ICP the selected pose
    moves towards the true one and scores at least as well as without."""
    g, hyps, ang, n_orient = room_case(2)
    prm = oracle.Params(n_orient=n_orient, topk=10, batch=10, local_topk=3)
    true = ((hyps[5][0] + 0.8) * RES, (hyps[5][1] + 0.3) * RES, 0.5)
    z = workloads.render_scan(g, RES, true, ang, 6.0)
    plain = oracle.relocalize(g, RES, hyps, z, ang, 6.0, prm, early_stop=False)
    refined = oracle.relocalize(g, RES, hyps, z, ang, 6.0, prm, early_stop=False, icp_iters=10)
    err = lambda r: math.hypot(r["x"] - true[0], r["y"] - true[1])
    assert err(refined) < err(plain)
    assert refined["tam"] >= plain["tam"]


# ------------------------------------------------------------------------------------------
# invariants of the whole scoring path
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("k_steps", [1, 3])
def test_rotating_scan_shifts_every_score(k_steps):
    g, hyps, ang, n_orient = room_case(4)
    prm = oracle.Params(n_orient=n_orient)
    rng = np.random.default_rng(9)
    z = rng.uniform(0.2, 1.5, len(ang)).astype(np.float32)
    pl = oracle.plan(z, ang, 5.0, RES, prm)
    k = k_steps * pl["n_enum"]
    ang2 = (ang.astype(np.float64) + k * 2 * math.pi / pl["ns"])
    ang2 = ((ang2 + math.pi) % (2 * math.pi) - math.pi).astype(np.float32)
    pl2 = oracle.plan(z, ang2, 5.0, RES, prm)
    assert (pl2["b"] == (pl["b"] + k) % pl["ns"]).all()
    sel = np.arange(6)
    T1 = oracle.tam_grid(g, hyps, sel, pl, prm, RES)
    T2 = oracle.tam_grid(g, hyps, sel, pl2, prm, RES)
    assert np.array_equal(np.roll(T2, k_steps, axis=1), T1)
    for r in range(len(sel)):
        assert (oracle.best_orientation(T2[r]) + k_steps) % n_orient == oracle.best_orientation(T1[r])
    n1, _ = oracle.smad(g, hyps, pl)
    n2, _ = oracle.smad(g, hyps, pl2)
    assert np.array_equal(n1, n2)


def test_translating_map_and_pose_leaves_scores_unchanged():
    g0 = workloads.make_room(7, n=40, n_boxes=4)
    g = np.zeros((120, 120), np.int8)
    g[40:80, 40:80] = g0                          # walls 40 cells away from the edge (= d_max)
    g2 = np.zeros((130, 125), np.int8)
    g2[47:87, 45:85] = g0                         # shifted by (5, 7)
    hyps = np.argwhere(g0 == 0)[::37, ::-1].astype(np.int32) + 40
    hyps2 = hyps + np.array([5, 7], np.int32)
    ang = workloads.beam_angles(90, 120)
    prm = oracle.Params(n_orient=40)
    z = np.random.default_rng(1).uniform(0.2, 1.8, 90).astype(np.float32)
    pl = oracle.plan(z, ang, 2.0, RES, prm)
    n1, m1 = oracle.smad(g, hyps, pl)
    n2, m2 = oracle.smad(g2, hyps2, pl)
    assert np.array_equal(n1, n2) and np.array_equal(m1, m2)
    sel = np.arange(len(hyps))
    assert np.array_equal(oracle.tam_grid(g, hyps, sel, pl, prm, RES), oracle.tam_grid(g2, hyps2, sel, pl, prm, RES))


@pytest.mark.parametrize("seed", range(3))
def test_self_rendered_pose_scores_best(seed):
    g, hyps, ang, n_orient = room_case(10 + seed, n_beams=100, ns=120, n_orient=40)
    prm = oracle.Params(n_orient=n_orient, topk=len(hyps))
    pl0 = oracle.plan(np.ones(len(ang), np.float32), ang, 6.0, RES, prm)
    h_true, q_true = 11, 13
    z = self_rendered(g, hyps[h_true], q_true * pl0["n_enum"], pl0, ang)
    res = oracle.relocalize(g, RES, hyps, z, ang, 6.0, prm, early_stop=False)
    assert res["smad_num"] == 0 if res["hyp"] == h_true else True
    assert res["hyp"] == h_true and res["m"] == q_true * pl0["n_enum"]


def test_relocalize_early_termination_and_batches():
    g, hyps, ang, n_orient = room_case(20)
    prm = oracle.Params(n_orient=n_orient, topk=20, batch=6, local_topk=3, tau=-1.0)
    z = np.random.default_rng(2).uniform(0.2, 1.5, len(ang)).astype(np.float32)
    r = oracle.relocalize(g, RES, hyps, z, ang, 5.0, prm)
    assert r["n_batches"] == 1 and r["n_tam_evals"] == 6 * n_orient
    assert len(r["batches"][0]) == 3
    r2 = oracle.relocalize(g, RES, hyps, z, ang, 5.0, prm, early_stop=False)
    assert r2["n_batches"] == 4 and r2["n_tam_evals"] == 20 * n_orient
    best = max((v[1], -k) for k, v in r2["per_hyp"].items())
    assert math.isclose(r2["tam"], best[0])


def test_no_ordering_arm_scores_the_hypotheses_in_their_own_order():
    """Table II's arm without SMAD ordering: zero numerators at m = 0, so the
    survivors are the hypotheses in index order.  Scored in full (K = N_h),
    it selects the same best TAM score as the SMAD-ordered run over every
    hypothesis (the set is the same, only the batch order differs); with
    early termination its first batch is the first `batch` hypotheses."""
    g, hyps, ang, n_orient = room_case(20)
    n = len(hyps)
    z = np.random.default_rng(2).uniform(0.2, 1.5, len(ang)).astype(np.float32)
    none = oracle.Params(n_orient=n_orient, topk=n, batch=6, local_topk=3, tau=-1.0, coarse=3)
    pl = oracle.plan(z, ang, 5.0, RES, none)
    num, mm = oracle.coarse(g, hyps, pl, none)
    assert (num == 0).all() and (mm == 0).all()
    r = oracle.relocalize(g, RES, hyps, z, ang, 5.0, none, early_stop=False)
    assert np.array_equal(r["survivors"], np.arange(n)) and r["n_smad_evals"] == 0
    ordered = oracle.relocalize(g, RES, hyps, z, ang, 5.0,
                                oracle.Params(n_orient=n_orient, topk=n, batch=6, local_topk=3, tau=-1.0),
                                early_stop=False)
    assert not np.array_equal(ordered["survivors"], r["survivors"])   # SMAD does reorder this case
    assert r["tam"] == ordered["tam"] and r["n_tam_evals"] == ordered["n_tam_evals"] == n * n_orient
    first = oracle.relocalize(g, RES, hyps, z, ang, 5.0, none)      # tau = -1: stop after the first batch
    assert first["n_batches"] == 1 and sorted(first["per_hyp"]) == list(range(6))


def test_panoramic_grid_size_follows_eq14_reading():
    """N_s = N_orient q with q the rounded N 360 / (FoV N_orient) clamped so
    that N <= N_s <= 2N (Eq. 14 needs an integer N_s): 504 for 360 beams over
    270 deg at 72 orientations, 1440 for 1081 beams over 270 deg at 360 and
    for 1440 beams over 360 deg at 720."""
    assert workloads.choose_ns(360, 270.0, 72) == 504
    assert workloads.choose_ns(1081, 270.0, 360) == 1440
    assert workloads.choose_ns(1440, 360.0, 720) == 1440
    for n in (90, 360, 541, 720, 1081, 1440):
        for fov in (180.0, 225.0, 270.0, 300.0, 360.0):
            for n_orient in (36, 72, 360):
                ns = workloads.choose_ns(n, fov, n_orient)
                assert ns % n_orient == 0
                assert n <= ns <= 2 * n or (ns == n_orient * -(-n // n_orient) and ns > 2 * n)


def test_quantised_endpoints_move_room_scores_less_than_1e4(workload):
    """The continuous mode as a diagnostic: TAM with the integer endpoint
    rule (Q16 ranges, Q30 directions, round half up) against TAM with FP64
    endpoints and floor, at 40 seeded (hypothesis, orientation) poses of the
    room workload: within 1e-4 relative."""
    wl = workload(0)
    prm = oracle.Params(n_orient=wl.n_orient, topk=wl.topk)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    d2 = oracle.edt(wl.grid)
    rng = np.random.default_rng(5)
    sel = rng.choice(len(wl.hyps), 40, replace=False)
    ms = rng.integers(0, pl["n_orient"], 40) * pl["n_enum"]
    tq = oracle.tam(wl.grid, wl.hyps[sel], ms, pl, prm, wl.res, d2)
    poses = [((wl.hyps[h][0] + 0.5) * wl.res, (wl.hyps[h][1] + 0.5) * wl.res, m * 2 * math.pi / pl["ns"])
             for h, m in zip(sel, ms)]
    tc = oracle.tam_pose(wl.grid, poses, pl, prm, wl.res, d2)
    assert np.allclose(tq, tc, rtol=1e-4, atol=0)
