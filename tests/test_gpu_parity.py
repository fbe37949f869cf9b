"""GPU path vs the CPU oracle, through the C ABI.

Bit-exact: EDT d2, clamped field and occupancy; synthesized ranges and hit
cells; SMAD numerators and minimising shifts; the SMAD survivor list; the
per-batch local top-k (up to TAM ties); counters.  Floating point: every TAM
score within 1e-5 relative of the FP64 oracle (the float32 epilogue's error
budget is about 1.5e-6: float32 table entries, a per-lane then shuffle-tree
top-k sum, and a cube root that divides the product's relative error by 3);
the selected pose identical unless the oracle scores the two candidates
within 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-5
RES = 0.05


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


def torch_():
    import torch
    return torch


def run(relo, grid, res, hyps, ranges, angles, max_range, **params):
    ctx = relo.Relo(**params)
    mid = ctx.load_map(grid, res)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, res))
    out = ctx.relocalize(mid, ranges, angles, max_range)
    return ctx, mid, out


def stages(relo, ctx, n_hyp, K, n_orient, n_batches, local_topk):
    torch = torch_()
    num = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(n_hyp, dtype=torch.int64, device="cuda")).cpu().numpy()
    mm = ctx.stage(relo.STAGE_SMAD_M, torch.empty(n_hyp, dtype=torch.int32, device="cuda")).cpu().numpy()
    surv = ctx.stage(relo.STAGE_SURVIVORS, torch.empty(K, dtype=torch.int32, device="cuda")).cpu().numpy()
    T = ctx.stage(relo.STAGE_TAM, torch.empty(K * n_orient, dtype=torch.float32, device="cuda")).cpu().numpy()
    bm = ctx.stage(relo.STAGE_BEST_M, torch.empty(K, dtype=torch.int32, device="cuda")).cpu().numpy()
    loc = ctx.stage(relo.STAGE_LOCAL_TOPK, torch.empty(n_batches * local_topk, dtype=torch.int32,
                                                       device="cuda")).cpu().numpy()
    info = ctx.stage(relo.STAGE_SCAN_INFO, torch.empty(relo.SCAN_INFO_LEN, dtype=torch.int64,
                                                       device="cuda")).cpu().numpy()
    return dict(num=num, m=mm, surv=surv, T=T.reshape(K, n_orient), best_m=bm,
                local=loc.reshape(n_batches, local_topk), info=info)


def assert_tam_close(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
    bad = ~((np.abs(got - want) <= RTOL * np.abs(want)) | ((want == 0) & (np.abs(got) <= 1e-7)))
    assert not bad.any(), f"{bad.sum()} TAM scores off; worst rel {err.max():.3g}"


def check_pose(got, want_hyp, want_m, T_or_fn):
    """Selected pose equal, or the oracle scores both candidates within RTOL."""
    if (got.hyp, got.m) == (want_hyp, want_m):
        return
    t_got, t_want = T_or_fn(got.hyp, got.m), T_or_fn(want_hyp, want_m)
    assert abs(t_got - t_want) <= RTOL * t_want, ((got.hyp, got.m, t_got), (want_hyp, want_m, t_want))


# ------------------------------------------------------------------------------------------
# EDT tables
# ------------------------------------------------------------------------------------------

def edt_case(relo, grid, res=0.05, d_max=2.0):
    torch = torch_()
    ctx = relo.Relo(d_max=d_max)
    mid = ctx.load_map(grid, res)
    d2, fld, occ = ctx.map_tables(mid, grid.shape)
    want = oracle.edt(grid)
    C = int(round(d_max / res)) ** 2
    assert np.array_equal(d2.cpu().numpy().astype(np.int64), want)
    assert np.array_equal(fld.cpu().numpy(), np.where((want < 0) | (want > C), C, want))
    assert np.array_equal(occ.cpu().numpy(), (grid >= 65).astype(np.uint8))
    ctx.close()


@pytest.mark.parametrize("shape,p", [((37, 53), 0.05), ((8, 8), 0.3), ((1, 1), 0.0), ((65, 1), 0.1),
                                     ((1, 77), 0.1), ((129, 200), 0.0), ((300, 257), 0.002)])
def test_edt_random_grids(relo, shape, p):
    rng = np.random.default_rng(hash(shape) % 2 ** 32)
    g = np.where(rng.random(shape) < p, 100, 0).astype(np.int8)
    g[rng.random(shape) < 0.03] = -1
    edt_case(relo, g)


def test_edt_room_and_office(relo, workload):
    edt_case(relo, workload(0).grid)
    edt_case(relo, workload(1).grid)


def test_edt_warehouse_sampled(relo, workload):
    torch = torch_()
    wl = workload(2)
    ctx = relo.Relo()
    mid = ctx.load_map(wl.grid, wl.res)
    d2, fld, occ = ctx.map_tables(mid, wl.grid.shape)
    want = oracle.edt(wl.grid)
    assert np.array_equal(d2.cpu().numpy().astype(np.int64), want)
    rng = np.random.default_rng(5)
    for _ in range(200):        # spot checks against the plain definition
        x, y = int(rng.integers(4096)), int(rng.integers(4096))
        assert d2[y, x].item() == oracle.d2_capped(wl.grid, x, y, 1 << 40)
    ctx.close()


# ------------------------------------------------------------------------------------------
# synthesized scans
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("cfg,n_check", [(0, 200), (1, 40), (2, 12)])
def test_synth_scans_bit_exact(relo, workload, cfg, n_check):
    torch = torch_()
    wl = workload(cfg)
    prm = oracle.Params(n_orient=wl.n_orient)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    ctx = relo.Relo(n_orient=wl.n_orient)
    mid = ctx.load_map(wl.grid, wl.res)
    sel = np.random.default_rng(cfg).choice(len(wl.hyps), n_check, replace=False)
    cells = torch.tensor(wl.hyps[sel], dtype=torch.int32, device="cuda")
    r, h = ctx.synth_scans(mid, cells, wl.angles, wl.max_range, pl["ns"])
    r, h = r.cpu().numpy().view(np.uint32), h.cpu().numpy()
    W = wl.grid.shape[1]
    for k, i in enumerate(sel):
        want_r, hx, hy = oracle.synth_scan(wl.grid, int(wl.hyps[i, 0]), int(wl.hyps[i, 1]), pl)
        assert np.array_equal(r[k].astype(np.int64), want_r)
        assert np.array_equal(h[k], np.where(hx < 0, -1, hy * W + hx))
    ctx.close()


# ------------------------------------------------------------------------------------------
# the whole path
# ------------------------------------------------------------------------------------------

def full_case(relo, wl, K, early_stop=False, batch=200, local_topk=20, tau=0.95, n_skip=1, sample_tam=None,
              d_max=2.0, coarse=0, fine=0, gpu_coarse=None):
    """The whole path against the oracle; gpu_coarse (default: coarse) is the
    library's ranking-metric code where it differs from the oracle's (the
    direct-window-sum SMAD is the oracle's SMAD, code 0)."""
    prm = oracle.Params(n_orient=wl.n_orient, topk=K, batch=batch, local_topk=local_topk, tau=tau,
                        n_skip_beam=n_skip, d_max=d_max, coarse=coarse, fine=fine)
    ctx, mid, got = run(relo, wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, n_orient=wl.n_orient,
                        topk=K, batch=batch, local_topk=local_topk, tau=tau, early_stop=int(early_stop),
                        n_skip_beam=n_skip, d_max=d_max, coarse_metric=coarse if gpu_coarse is None else gpu_coarse,
                        fine_metric=fine)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    Kc = min(K, len(wl.hyps))
    B = min(batch, Kc)
    nb = -(-Kc // B)
    st = stages(relo, ctx, len(wl.hyps), Kc, pl["n_orient"], nb, local_topk)
    # SMAD (or CAER) and ranking: bit-exact
    num, mm = oracle.coarse(wl.grid, wl.hyps, pl, prm)
    assert np.array_equal(st["num"], num)
    assert np.array_equal(st["m"], mm)
    surv = oracle.rank(num, Kc)
    assert np.array_equal(st["surv"], surv)
    info = st["info"]
    assert info[0] == pl["ns"] and info[1] == pl["n_orient"] and info[3] == pl["n_valid"]
    assert info[5] == pl["sum_real"] and info[6] == Kc
    k_ret = sorted([pl["n_valid"], max(1, math.floor(pl["a_mid"] * pl["n_valid"])),
                    max(1, math.floor(pl["a_low"] * pl["n_valid"]))])[1]
    assert info[4] == k_ret
    d2 = oracle.edt(wl.grid)
    n_scored = int(info[7]) * B
    n_scored = min(n_scored, Kc)
    rows = np.arange(n_scored) if sample_tam is None else np.unique(np.concatenate(
        [np.random.default_rng(1).choice(n_scored, min(sample_tam, n_scored), replace=False), [0]]))
    T_or = oracle.tam_grid(wl.grid, wl.hyps, surv[rows], pl, prm, wl.res, d2)
    assert_tam_close(st["T"][rows], T_or)
    assert np.isnan(st["T"][n_scored:]).all()
    # orientation argmax per scored survivor (Eq. 22)
    for r_i, r in enumerate(rows):
        q_or = oracle.best_orientation(T_or[r_i])
        q_gpu = st["best_m"][r] // pl["n_enum"]
        if q_gpu != q_or:
            assert abs(T_or[r_i, q_gpu] - T_or[r_i, q_or]) <= RTOL * T_or[r_i, q_or]
    assert got.status == 0 and got.n_batches == info[7]
    assert got.n_tam_evals == n_scored * pl["n_orient"]
    assert got.n_smad_evals == (0 if coarse == 3 else len(wl.hyps) * (1 if pl["panoramic"] else pl["n_orient"]))
    return ctx, got, st, pl, prm, d2, surv, rows, T_or


@pytest.mark.parametrize("cfg", [0, 1])
def test_full_path_matches_oracle(relo, workload, cfg):
    wl = workload(cfg)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk)
    want = oracle.relocalize(wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range,
                             oracle.Params(n_orient=wl.n_orient, topk=wl.topk), d2tab=d2, early_stop=False)

    def T_at(h, m):
        return float(oracle.tam(wl.grid, np.array([wl.hyps[h]]), np.array([m]), pl, prm, wl.res, d2)[0])
    check_pose(got, want["hyp"], want["m"], T_at)
    assert abs(got.tam - T_at(got.hyp, got.m)) <= RTOL * T_at(got.hyp, got.m)
    assert math.isclose(got.x, (wl.hyps[got.hyp, 0] + 0.5) * wl.res) and got.smad_num == st["num"][got.hyp]
    th = got.m * 2 * math.pi / pl["ns"]
    assert math.isclose(got.theta, th - 2 * math.pi if th >= math.pi else th, abs_tol=1e-12)
    ctx.close()


@pytest.mark.parametrize("gap", [0, 14])
def test_single_orientation_smad_paths(relo, workload, gap):
    """SMAD with one orientation (m = 0, lambda >= 0.9, Eq. 20) sums each row
    over the FoV intervals directly (one interval of every direction, or two
    around a gap); with resident synthesized scans W_0 comes from window tables
    built from the stored rows.  Every numerator equals the oracle's."""
    torch = torch_()
    wl = workload(0)
    ns = 504
    ang = workloads.beam_angles(ns, ns)
    keep = np.ones(ns, bool)
    keep[100:100 + gap] = False
    ang = ang[keep]
    pose = (wl.hyps[7, 0], wl.hyps[7, 1], 0.0)
    z = workloads.render_scan(wl.grid, wl.res, ((pose[0] + 0.5) * wl.res, (pose[1] + 0.5) * wl.res, 0.0), ang,
                              wl.max_range)
    prm = oracle.Params(n_orient=wl.n_orient, topk=16)
    pl = oracle.plan(z, ang, wl.max_range, wl.res, prm)
    assert pl["ns"] == ns and pl["lam"] >= 0.9
    num, mm = oracle.coarse(wl.grid, wl.hyps, pl, prm)
    runs = []
    for cache in (0, 64 << 20, 64 << 20):   # no resident scans; then a request that stores them, one that reads
        if cache == 0 or len(runs) == 1:
            if runs:
                ctx.close()
            ctx = relo.Relo(n_orient=wl.n_orient, topk=16, early_stop=0, scan_cache_bytes=cache)
            mid = ctx.load_map(wl.grid, wl.res)
            ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
        out = ctx.relocalize(mid, z, ang, wl.max_range)
        assert out.status == 0
        got = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(wl.hyps), dtype=torch.int64, device="cuda")).cpu()
        assert np.array_equal(got.numpy(), num) and not mm.any()
        runs.append(cache)
    ctx.close()


@pytest.mark.parametrize("d_max", [2.2, 2.25, 2.3, 3.85, 3.9, 3.95, 4.5])
def test_selection_counts_either_side_of_fp16_range(relo, workload, d_max):
    """The TAM selection counts run on packed fp16 patterns 0x6400 + s, s the
    table slot b + floor(b / 32) of the clamped value b, while the slot of
    C + 1 is at most 6143 (d_max / res = 77: C = 5929, slot 6115), and in
    32-bit integers above (78^2 = 6084, slot 6275; 79^2 = 6241; 90^2 = 8100,
    the largest clamp).  44 and 45 put the largest slot either side of 2048
    (45 and 46 the largest value), where the fp16 numbers of consecutive
    patterns go from 2 to 4 apart.  All match the oracle."""
    wl = workload(0)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk, d_max=d_max)
    want = oracle.relocalize(wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, prm, d2tab=d2,
                             early_stop=False)

    def T_at(h, m):
        return float(oracle.tam(wl.grid, np.array([wl.hyps[h]]), np.array([m]), pl, prm, wl.res, d2)[0])
    check_pose(got, want["hyp"], want["m"], T_at)
    ctx.close()


@pytest.mark.parametrize("fine", [1, 2, 3])
def test_fine_metrics_match_oracle(relo, workload, fine):
    """TAM_mean (Eq. 34), wp_baseline (Eq. 33) and wp_LF (Eq. 32, negative
    sums) scored in place of TAM: every score within 1e-5 of the oracle's
    magnitude, the orientation argmax, and the selected pose."""
    wl = workload(0)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk, fine=fine)
    want = oracle.relocalize(wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, prm, d2tab=d2,
                             early_stop=False)

    def T_at(h, m):
        return float(oracle.tam(wl.grid, np.array([wl.hyps[h]]), np.array([m]), pl, prm, wl.res, d2)[0])
    check_pose(got, want["hyp"], want["m"], T_at)
    if fine == 3:
        assert got.tam < 0
    ctx.close()


def test_caer_ranking_matches_oracle(relo, workload):
    """CAER (Eq. 21) in place of SMAD: numerators, minimising m and the
    survivor list bit-exact; TAM on those survivors within tolerance."""
    wl = workload(0)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk, coarse=1)
    assert not pl["panoramic"]
    sn, _ = oracle.smad(wl.grid, wl.hyps, pl)
    assert np.all(st["num"] >= sn)   # Eq. 21 bounds Eq. 19 at every m
    ctx.close()


def test_caer_panoramic_and_fine_metric_together(relo):
    """A full-circle scan (Eq. 20: m = 0 only) ranked by CAER and scored by
    wp_baseline, with early termination."""
    wl = small_case(n_beams=120, ns=120)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, 12, batch=4, local_topk=2, coarse=1, fine=2,
                                                             early_stop=True, tau=0.5)
    assert pl["panoramic"] and (st["m"] == 0).all()
    ctx.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_smad_by_direct_window_sums_matches_oracle(relo, workload, cfg):
    """SMAD with every Eq. 18 window sum added up position by position (no
    Eq. 17 prefix sums, the Table II ablation): numerators, minimising m and
    the survivor list bit-exact against the oracle, whose SMAD is that form;
    the selected pose as with the prefix sums."""
    wl = workload(cfg)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk, coarse=0, gpu_coarse=2,
                                                             sample_tam=None if cfg == 0 else 6)
    ctx.close()
    ctx2, _, ref = run(relo, wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, n_orient=wl.n_orient,
                       topk=wl.topk, early_stop=0)
    assert (got.hyp, got.m, got.smad_num) == (ref.hyp, ref.m, ref.smad_num) and got.tam == ref.tam
    ctx2.close()


def test_smad_by_direct_window_sums_panoramic_and_ragged(relo):
    """The direct form on a full-circle scan (Eq. 20: m = 0 only) and on a
    partial scan whose FoV wraps past beam 0, with early termination."""
    for n_beams, ns in ((120, 120), (90, 120)):
        wl = small_case(n_beams=n_beams, ns=ns)
        ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, 12, batch=4, local_topk=2, coarse=0,
                                                                 gpu_coarse=2, early_stop=True, tau=0.5)
        assert pl["panoramic"] == (n_beams == ns)
        ctx.close()


@pytest.mark.parametrize("early,tau", [(False, 0.95), (True, 0.5)])
def test_no_ordering_arm_matches_oracle(relo, workload, early, tau):
    """Table II's arm without SMAD ordering: zero numerators at m = 0, every
    hypothesis a survivor in its own order, then TAM batch by batch with the
    local top-k and early termination as the oracle takes them."""
    wl = workload(0)
    n = len(wl.hyps)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, n, batch=50, local_topk=5, coarse=3,
                                                             early_stop=early, tau=tau)
    assert (st["num"] == 0).all() and (st["m"] == 0).all()
    assert np.array_equal(st["surv"], np.arange(n))
    want = oracle.relocalize(wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, prm, d2tab=d2,
                             early_stop=early)
    assert got.n_batches == want["n_batches"] and (early or got.n_batches == -(-n // 50))

    def T_at(h, m):
        return float(oracle.tam(wl.grid, np.array([wl.hyps[h]]), np.array([m]), pl, prm, wl.res, d2)[0])
    check_pose(got, want["hyp"], want["m"], T_at)
    ctx.close()


def edge_margin(pl, pose, res=RES):
    """Smallest distance, in cells, from a valid beam's world point at a
    continuous pose (x + z cos(theta + a), y + z sin(theta + a)) to a cell
    edge.  Where it is tiny the containing cell depends on rounding, and two
    correct programs may put the point in either neighbour."""
    z, a = oracle.scan_points(pl, res)
    w = np.concatenate([(pose[0] + z * np.cos(pose[2] + a)) / res, (pose[1] + z * np.sin(pose[2] + a)) / res])
    f = w - np.floor(w)
    return float(np.minimum(f, 1.0 - f).min())


def icp_case(relo, g, hyps, z, ang, max_range, early, **kw):
    """ICP (10 iterations) of every local top-k pose through the library
    against the oracle's plain arithmetic.  The scans are noisy, so no beam
    ends on a cell edge at either refined pose; the test checks that margin,
    without which the two cell assignments (and with them the pairs and the
    scores) could legitimately differ."""
    prm = oracle.Params(n_orient=kw.get("n_orient", 40), topk=kw.get("topk", 12), batch=kw.get("batch", 6),
                        local_topk=kw.get("local_topk", 3), tau=kw.get("tau", 0.95))
    d2 = oracle.edt(g)
    want = oracle.relocalize(g, RES, hyps, z, ang, max_range, prm, d2tab=d2, early_stop=early, icp_iters=10)
    ctx, mid, got = run(relo, g, RES, hyps, z, ang, max_range, n_orient=prm.n_orient, topk=prm.topk, batch=prm.batch,
                        local_topk=prm.local_topk, tau=prm.tau, early_stop=int(early), icp_iters=10)
    ctx.close()
    assert got.status == 0 and got.n_batches == want["n_batches"]
    pl = want["plan"]
    assert edge_margin(pl, (want["x"], want["y"], want["theta"])) > 1e-6
    assert edge_margin(pl, (got.x, got.y, got.theta)) > 1e-6
    if (got.hyp, got.m) == (want["hyp"], want["m"]):
        dth = math.remainder(got.theta - want["theta"], 2 * math.pi)
        assert abs(got.x - want["x"]) <= 1e-6 and abs(got.y - want["y"]) <= 1e-6 and abs(dth) <= 1e-6
    assert abs(got.tam - want["tam"]) <= RTOL * abs(want["tam"])
    return got, want


@pytest.mark.parametrize("early", [False, True])
def test_icp_refinement_matches_oracle(relo, early):
    """ICP of every local top-k pose (10 iterations) and its re-evaluation at
    the refined continuous pose: the selected hypothesis, orientation and
    refined pose equal the oracle's (1e-6 m and rad), the re-evaluated score
    within 1e-5; a scan rendered between cells with 5 mm range noise, with and
    without early termination."""
    g = workloads.make_room(2, n=40, n_boxes=4)
    free = np.argwhere(g == 0)[:, ::-1]
    hyps = free[np.random.default_rng(2).choice(len(free), 25, replace=False)].astype(np.int32)
    ang = workloads.beam_angles(90, 120)
    true = ((hyps[5][0] + 0.8) * RES, (hyps[5][1] + 0.3) * RES, 0.5)
    z = workloads.add_noise(workloads.render_scan(g, RES, true, ang, 6.0), 6.0, 5, sigma=0.005, drop_frac=0.0,
                            short_frac=0.0)
    got, want = icp_case(relo, g, hyps, z, ang, 6.0, early, tau=0.5)
    plain = oracle.relocalize(g, RES, hyps, z, ang, 6.0, oracle.Params(n_orient=40, topk=12, batch=6, local_topk=3,
                                                                       tau=0.5), early_stop=early)
    assert math.hypot(got.x - true[0], got.y - true[1]) < math.hypot(plain["x"] - true[0], plain["y"] - true[1])


def test_icp_on_the_room_workload(relo, workload):
    """The room workload's scan (noise-free by definition) with 5 mm range
    noise added, so that no endpoint sits on a cell edge."""
    wl = workload(0)
    z = workloads.add_noise(wl.ranges, wl.max_range, 6, sigma=0.005, drop_frac=0.0, short_frac=0.0)
    icp_case(relo, wl.grid, wl.hyps, z, wl.angles, wl.max_range, False, n_orient=wl.n_orient, topk=16,
             batch=8, local_topk=4)


@pytest.mark.parametrize("fine", [0, 1, 2, 3])
def test_translation_sweep_matches_oracle(relo, workload, fine):
    """The Fig. 8 sweep in kind (office workload): 15 cells 0.1 m apart through
    the scan's true position x 36 orientations 10 degrees apart, scored by
    each scoring metric (TAM, TAM_mean, wp_baseline, wp_LF) through the library
    as bench.py's sweep runs it; every one of the 540 scores equals the
    oracle's at the same pose within 1e-5 (of its magnitude)."""
    torch = torch_()
    wl = workload(1)
    cells, offs, axis, qs = workloads.sweep_poses(wl)
    ctx = relo.Relo(n_orient=360, topk=len(cells), batch=len(cells), local_topk=1, early_stop=0, fine_metric=fine)
    mid = ctx.load_map(wl.grid, wl.res)
    ctx.set_hypotheses(mid, workloads.cell_centres(cells, wl.res))
    got = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert got.status == relo.OK
    surv = ctx.stage(relo.STAGE_SURVIVORS, torch.empty(len(cells), dtype=torch.int32, device="cuda")).cpu().numpy()
    T = ctx.stage(relo.STAGE_TAM, torch.empty(len(cells) * 360, dtype=torch.float32, device="cuda"))
    ctx.close()
    rows = np.empty((len(cells), 360), np.float32)
    rows[surv] = T.cpu().numpy().reshape(len(cells), 360)
    prm = oracle.Params(n_orient=360, topk=len(cells))
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    d2 = oracle.edt(wl.grid)
    pairs = np.repeat(cells, len(qs), axis=0)
    ms = np.tile(np.array(qs, np.int32) * pl["n_enum"], len(cells))
    want = oracle.tam(wl.grid, pairs, ms, pl, prm, wl.res, d2, metric=fine).reshape(len(cells), len(qs))
    assert_tam_close(rows[:, qs], want)


def test_warehouse_full_size_sampled(relo, workload):
    """4096^2 map, 20000 hypotheses, 720 orientations, K = 1024: SMAD and the
    survivor list bit-exact everywhere; TAM on 48 sampled survivors x 720."""
    wl = workload(2)
    ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, wl.topk, sample_tam=48)
    assert pl["panoramic"]                    # 360-degree scan: SMAD at m = 0 only (Eq. 20)
    # the selected pose scores at least as well as every sampled survivor's best
    T_sel = float(oracle.tam(wl.grid, np.array([wl.hyps[got.hyp]]), np.array([got.m]), pl, prm, wl.res, d2)[0])
    assert abs(got.tam - T_sel) <= RTOL * T_sel
    assert T_sel >= T_or.max() * (1 - RTOL)
    ctx.close()


def test_batches_early_termination_and_local_topk(relo, workload):
    wl = workload(1)
    for tau, early in ((0.0, True), (2.0, True), (0.95, False)):
        ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl, 100, early_stop=early, batch=30,
                                                                 local_topk=7, tau=tau)
        want = oracle.relocalize(wl.grid, wl.res, wl.hyps, wl.ranges, wl.angles, wl.max_range, prm, d2tab=d2,
                                 early_stop=early)
        assert got.n_batches == want["n_batches"] == (1 if tau == 0.0 else 4)
        for b, local in enumerate(want["batches"]):
            g = [int(s) for s in st["local"][b] if s >= 0]
            w = [pos for (_, pos, _, _) in local]
            if g != w:   # allow swaps of TAM ties within tolerance
                Tg = [T_or[s].max() for s in g]
                Tw = [T_or[s].max() for s in w]
                assert np.allclose(Tg, Tw, rtol=RTOL)
        ctx.close()


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------

def small_case(seed=3, n_beams=90, ns=120, n_orient=40, max_range=4.0):
    g = workloads.make_room(seed, n=40, n_boxes=4)
    free = np.argwhere(g == 0)[:, ::-1]
    hyps = free[np.random.default_rng(seed).choice(len(free), 30, replace=False)].astype(np.int32)
    ang = workloads.beam_angles(n_beams, ns)
    z = workloads.render_scan(g, 0.05, ((hyps[4, 0] + 0.5) * 0.05, (hyps[4, 1] + 0.5) * 0.05, 0.3), ang, max_range)
    return workloads.Workload("small", g, 0.05, hyps, z, ang, max_range, n_orient, 8, ns, (0, 0, 0))


def test_ragged_batches_skip_and_topk_over_n(relo):
    wl = small_case()
    # 88 beams start on an even panoramic index, so every second beam (Eq. 11)
    # still lies on the coarser grid of N_s = 60 directions (Eq. 14)
    wl88 = small_case(n_beams=88)
    for K, batch, local, skip in ((8, 3, 2, 1), (64, 7, 3, 2), (1, 1, 1, 1)):
        wl2 = wl
        if skip > 1:   # n_orient must divide the downsampled N_s
            wl2 = workloads.Workload("small", wl88.grid, wl88.res, wl88.hyps, wl88.ranges, wl88.angles,
                                     wl88.max_range, 20, K, 60, wl88.gt_pose)
        ctx, got, st, pl, prm, d2, surv, rows, T_or = full_case(relo, wl2, K, batch=batch, local_topk=local,
                                                                 n_skip=skip)
        ctx.close()


def test_gapped_fov_two_intervals(relo):
    wl = small_case(n_beams=100, ns=120)
    keep = np.r_[0:30, 45:100]                 # an occluded sector (Eq. 12)
    wl = workloads.Workload("gap", wl.grid, wl.res, wl.hyps, wl.ranges[keep], wl.angles[keep], wl.max_range, 40, 10,
                            120, wl.gt_pose)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, oracle.Params(n_orient=40))
    assert pl["K"] == 2 and pl["ns"] == 120
    ctx, *_ = full_case(relo, wl, 10)
    ctx.close()


def test_errors_are_reported(relo):
    wl = small_case()
    ctx = relo.Relo(n_orient=40, topk=8)
    mid = ctx.load_map(wl.grid, wl.res)
    with pytest.raises(relo.ReloError) as e:
        ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert e.value.code == relo.E_NO_HYPOTHESES
    occ = np.argwhere(wl.grid >= 65)[0][::-1]
    with pytest.raises(relo.ReloError) as e:
        ctx.set_hypotheses(mid, workloads.cell_centres(occ[None].astype(np.int32), wl.res))
    assert e.value.code == relo.E_INVALID_ARG
    ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
    with pytest.raises(relo.ReloError) as e:
        ctx.relocalize(mid, np.full_like(wl.ranges, wl.max_range), wl.angles, wl.max_range)
    assert e.value.code == relo.E_NO_VALID_BEAMS
    bad = wl.angles.copy()
    bad[10] += 0.3 * 2 * math.pi / 120
    with pytest.raises(relo.ReloError) as e:
        ctx.relocalize(mid, wl.ranges, bad, wl.max_range)
    assert e.value.code == relo.E_BEAM_GRID
    with pytest.raises(relo.ReloError) as e:
        ctx.relocalize(mid + 5, wl.ranges, wl.angles, wl.max_range)
    assert e.value.code == relo.E_NOT_FOUND
    ok = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)      # context still usable
    assert ok.status == 0
    ctx.close()



def test_metre_hypotheses_snap_like_the_definition(relo):
    """relo_set_hypotheses snaps metre coordinates to cells on the device:
    cell = floor((x - origin) / res) per axis in FP64.  Points at cell
    centres, exactly on cell edges and just inside the far edge, with a
    nonzero origin, give the same per-hypothesis SMAD numerators (Eq. 19) as
    the cells numpy computes by that expression, passed as cells."""
    import torch
    wl = small_case()
    origin = (-1.3, 2.15)
    rng = np.random.default_rng(11)
    free = np.argwhere(wl.grid < 65)[:, ::-1]
    pick = free[rng.choice(len(free), 400, replace=False)].astype(np.float64)
    frac = rng.choice([0.0, 0.5, 0.25, 1.0 - 1e-9], size=pick.shape)
    xy = (pick + frac) * wl.res + np.array(origin)
    cells = np.floor((xy - np.array(origin)) / wl.res).astype(np.int64)
    H, W = wl.grid.shape
    ok = (cells[:, 0] >= 0) & (cells[:, 1] >= 0) & (cells[:, 0] < W) & (cells[:, 1] < H)
    ok[ok] &= wl.grid[cells[ok, 1], cells[ok, 0]] < 65
    xy, cells = xy[ok], cells[ok].astype(np.int32)
    assert len(xy) > 300
    nums = []
    for how in ("metres", "cells"):
        ctx = relo.Relo(n_orient=wl.n_orient, topk=8)
        mid = ctx.load_map(wl.grid, wl.res, origin)
        if how == "metres":
            ctx.set_hypotheses(mid, xy)
        else:
            ctx.set_hypotheses_cells_dev(mid, torch.tensor(cells, device="cuda"))
        ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
        nums.append(ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(xy), dtype=torch.int64, device="cuda")).cpu().numpy())
        ctx.close()
    assert np.array_equal(nums[0], nums[1])


@pytest.mark.parametrize("bad", ["off_map", "nan", "occupied"])
def test_bad_metre_hypotheses_leave_none(relo, bad):
    """An off-map, non-finite or occupied point fails the whole call with
    E_INVALID_ARG, and the map then has no hypotheses until a good call."""
    wl = small_case()
    ctx = relo.Relo(n_orient=wl.n_orient, topk=8)
    mid = ctx.load_map(wl.grid, wl.res)
    good = workloads.cell_centres(wl.hyps, wl.res)
    ctx.set_hypotheses(mid, good)
    xy = good.copy()
    if bad == "off_map":
        xy[7] = (-0.01, 0.3)
    elif bad == "nan":
        xy[3, 1] = np.nan
    else:
        occ = np.argwhere(wl.grid >= 65)[0][::-1]
        xy[5] = (occ + 0.5) * wl.res
    with pytest.raises(relo.ReloError) as e:
        ctx.set_hypotheses(mid, xy)
    assert e.value.code == relo.E_INVALID_ARG
    with pytest.raises(relo.ReloError) as e:
        ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert e.value.code == relo.E_NO_HYPOTHESES
    ctx.set_hypotheses(mid, good)
    assert ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range).status == 0
    ctx.close()

def test_degenerate_single_cell_map(relo):
    g = np.zeros((1, 1), np.int8)
    ang = workloads.beam_angles(8, 16)
    wl = workloads.Workload("1x1", g, 0.05, np.zeros((1, 2), np.int32), np.full(8, 0.5, np.float32), ang, 3.0, 8, 1,
                            16, (0, 0, 0))
    ctx, got, st, pl, *_ = full_case(relo, wl, 1)
    assert got.tam == 0.0 and got.m == 0 and got.hyp == 0
    ctx.close()


def test_device_entry_points_match_host_ones(relo, workload):
    torch = torch_()
    wl = workload(0)
    ctx = relo.Relo(n_orient=wl.n_orient, topk=wl.topk, early_stop=0)
    g = torch.tensor(wl.grid, device="cuda")
    mid = ctx.load_map_dev(g, wl.res)
    ctx.set_hypotheses_cells_dev(mid, torch.tensor(wl.hyps, device="cuda"))
    z = torch.tensor(wl.ranges, device="cuda")
    res = torch.empty(relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.relocalize_dev(mid, z, wl.angles, wl.max_range, res)
    torch.cuda.synchronize()
    got = relo.result_from_bytes(bytes(res.cpu().numpy()))
    host = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert got.as_dict() == host.as_dict()
    ctx.update_map_dev(mid, g)                  # same grid: same answer
    again = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert again.as_dict() == host.as_dict()
    ctx.close()


def test_host_entry_points_repeated(relo, workload):
    """The end-to-end loop of the benchmark: map, hypotheses and scan re-sent
    from pinned host buffers every call, identical results each time."""
    torch = torch_()
    wl = workload(1)
    ctx = relo.Relo(n_orient=wl.n_orient, topk=wl.topk, early_stop=0)
    mid = ctx.load_map(wl.grid, wl.res)
    grid_h = torch.from_numpy(np.ascontiguousarray(wl.grid)).pin_memory()
    xy_h = torch.from_numpy(workloads.cell_centres(wl.hyps, wl.res)).pin_memory()
    z_h = torch.from_numpy(np.ascontiguousarray(wl.ranges)).pin_memory()
    out = relo.Result()
    first = None
    for _ in range(5):
        ctx.update_map_ptr(mid, grid_h.data_ptr())
        ctx.set_hypotheses_ptr(mid, xy_h.data_ptr(), len(wl.hyps))
        ctx.relocalize_ptr(mid, z_h.data_ptr(), wl.angles, len(wl.ranges), wl.max_range, out)
        d = out.as_dict()
        first = first or d
        assert d == first and d["status"] == 0
    ctx.close()


def test_profiling_then_blocking_call_then_close(relo, workload):
    """Stage timing on device steps, then the first blocking host-pointer call,
    then destroy: the context must tear down cleanly."""
    torch = torch_()
    wl = workload(0)
    ctx = relo.Relo(n_orient=wl.n_orient, topk=wl.topk, early_stop=0)
    g = torch.tensor(wl.grid, device="cuda")
    mid = ctx.load_map_dev(g, wl.res)
    ctx.set_hypotheses_cells_dev(mid, torch.tensor(wl.hyps, device="cuda"))
    z = torch.tensor(wl.ranges, device="cuda")
    res = torch.empty(relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.set_profiling(True)
    for _ in range(3):
        ctx.update_map_dev(mid, g)
        ctx.relocalize_dev(mid, z, wl.angles, wl.max_range, res)
    ms, n, k = ctx.stage_times(reset=True)
    ctx.set_profiling(False)
    # an EDT is timed in two parts: the occupancy tiles, then the field pass on the side stream
    assert n["raycast"] == 3 and n["smad"] == 3 and n["edt"] == 3 and n["edt_field"] == 3
    assert all(v >= 0 for v in ms.values()) and k > 0
    out = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range)
    assert out.status == 0
    ctx.close()


def mixed_batch_items(workload):
    """Requests on different maps with different sensors, FoVs and hypothesis counts."""
    items = []
    wl0 = workload(0)
    items.append((wl0.grid, wl0.res, wl0.hyps, wl0.ranges, wl0.angles, wl0.max_range, wl0.n_orient))
    g = workloads.make_office(77, n=256)
    hyps = np.argwhere(g == 0)[:, ::-1]
    hyps = hyps[np.random.default_rng(4).choice(len(hyps), 700, replace=False)].astype(np.int32)
    for n_beams, ns, seed in ((541, 720, 1), (720, 1080, 2), (360, 360, 3)):
        ang = workloads.beam_angles(n_beams, ns)
        h = hyps[seed * 5]
        z = workloads.render_scan(g, 0.05, ((h[0] + 0.5) * 0.05, (h[1] + 0.5) * 0.05, 0.7 * seed), ang, 12.0)
        z = workloads.add_noise(z, 12.0, seed)
        items.append((g, 0.05, hyps[: 300 * seed], z, ang, 12.0, 72 if ns != 360 else 72))
    wl = small_case(n_beams=100, ns=120)
    keep = np.r_[0:30, 45:100]
    items.append((wl.grid, wl.res, wl.hyps, wl.ranges[keep], wl.angles[keep], wl.max_range, 40))
    return items


def test_batch_equals_single_requests(relo, workload):
    items = mixed_batch_items(workload)
    # the orientation count is a context parameter: one context per count
    groups = {}
    for it in items:
        groups.setdefault(it[6], []).append(it)
    for n_orient, group in groups.items():
        ctx = relo.Relo(n_orient=n_orient, topk=32, batch=12, local_topk=4, early_stop=1, tau=0.9)
        reqs = []
        for (g, res, hyps, z, ang, mr, _) in group:
            mid = ctx.load_map(g, res)
            ctx.set_hypotheses(mid, workloads.cell_centres(hyps, res))
            reqs.append((mid, z, ang, mr))
        batch = ctx.relocalize_batch(reqs)
        for (mid, z, ang, mr), got in zip(reqs, batch):
            one = ctx.relocalize(mid, z, ang, mr)
            assert got.as_dict() == one.as_dict()
        ctx.close()


def test_cast_grouping_in_a_large_batch(relo, workload):
    """A batch with enough rays casts four hypotheses per work item, where the
    same office request alone casts two (the group size follows the batch's
    ray count): results equal the request alone, and the first request's SMAD
    numerators (Eq. 19) equal the oracle's."""
    torch = torch_()
    wl = workload(1)
    ctx = relo.Relo(n_orient=wl.n_orient, topk=wl.topk, early_stop=0)
    mid = ctx.load_map(wl.grid, wl.res)
    ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
    z2 = workloads.add_noise(wl.ranges, wl.max_range, 99)
    reqs = [(mid, wl.ranges, wl.angles, wl.max_range), (mid, z2, wl.angles, wl.max_range)]
    batch = ctx.relocalize_batch(reqs)
    got = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(wl.hyps), dtype=torch.int64, device="cuda")).cpu().numpy()
    prm = oracle.Params(n_orient=wl.n_orient, topk=wl.topk)
    pl = oracle.plan(wl.ranges, wl.angles, wl.max_range, wl.res, prm)
    num, _ = oracle.coarse(wl.grid, wl.hyps, pl, prm)
    assert np.array_equal(got, num)
    for (m, z, a, mr), b in zip(reqs, batch):
        assert b.as_dict() == ctx.relocalize(m, z, a, mr).as_dict()
    ctx.close()


def test_batch_dev_equals_host_and_oracle(relo, workload):
    torch = torch_()
    wl = workload(1)
    g2 = workloads.make_office(91, n=512)
    free = np.argwhere(g2 == 0)[:, ::-1]
    h2 = free[np.random.default_rng(8).choice(len(free), 1500, replace=False)].astype(np.int32)
    ang2 = workloads.beam_angles(1081, 1440)
    z2 = workloads.add_noise(workloads.render_scan(g2, 0.05, ((h2[9, 0] + 0.5) * 0.05, (h2[9, 1] + 0.5) * 0.05, 1.0),
                                                   ang2, 25.0), 25.0, 5)
    ctx = relo.Relo(n_orient=360, topk=64, early_stop=0)
    m1 = ctx.load_map(wl.grid, wl.res)
    ctx.set_hypotheses(m1, workloads.cell_centres(wl.hyps, wl.res))
    m2 = ctx.load_map(g2, 0.05)
    ctx.set_hypotheses(m2, workloads.cell_centres(h2, 0.05))
    items = [(m1, wl.ranges, wl.angles, wl.max_range), (m2, z2, ang2, 25.0), (m1, z2, ang2, 25.0)]
    host = ctx.relocalize_batch(items)
    res_t = torch.empty(len(items) * relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    dev_items = [(m, torch.tensor(z, device="cuda"), a, mr) for (m, z, a, mr) in items]
    ctx.relocalize_batch_dev(dev_items, res_t)
    torch.cuda.synchronize()
    raw = bytes(res_t.cpu().numpy())
    for i, h in enumerate(host):
        d = relo.result_from_bytes(raw[i * relo.RESULT_BYTES:(i + 1) * relo.RESULT_BYTES])
        assert d.as_dict() == h.as_dict()
    # the second request against the oracle
    prm = oracle.Params(n_orient=360, topk=64)
    want = oracle.relocalize(g2, 0.05, h2, z2, ang2, 25.0, prm, early_stop=False)
    pl = oracle.plan(z2, ang2, 25.0, 0.05, prm)
    d2 = oracle.edt(g2)

    def T_at(h, m):
        return float(oracle.tam(g2, np.array([h2[h]]), np.array([m]), pl, prm, 0.05, d2)[0])
    check_pose(host[1], want["hyp"], want["m"], T_at)
    assert abs(host[1].tam - T_at(host[1].hyp, host[1].m)) <= RTOL * T_at(host[1].hyp, host[1].m)
    assert host[1].smad_num == want["smad_nums"][host[1].hyp]
    ctx.close()


def served_setup(relo, workload, **params):
    items = [it for it in mixed_batch_items(workload) if it[6] == 72]
    ctx = relo.Relo(n_orient=72, topk=32, batch=12, local_topk=4, early_stop=1, tau=0.9, **params)
    reqs = []
    for (g, res, hyps, z, ang, mr, _) in items:
        mid = ctx.load_map(g, res)
        ctx.set_hypotheses(mid, workloads.cell_centres(hyps, res))
        reqs.append((mid, z, ang, mr))
    return ctx, reqs


def poll_all(ctx, tickets, timeout_s=60.0):
    import time
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = ctx.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout_s, "served requests did not finish"
        time.sleep(0.001)
    return [out[t] for t in tickets]


def test_served_results_equal_alone(relo, workload):
    """Continuous batching: a mixed stream of requests, submitted in waves
    while earlier ones run, gives every request the result it gets alone."""
    ctx, reqs = served_setup(relo, workload)
    alone = [ctx.relocalize(*r).as_dict() for r in reqs]
    ctx.serve_start(max_batch=3, max_inflight=2)
    order = [i % len(reqs) for i in range(17)]
    tickets = [ctx.submit(*reqs[i]) for i in order[:9]]
    tickets += [ctx.submit(*reqs[i]) for i in order[9:]]
    done = poll_all(ctx, tickets)
    ctx.serve_stop()
    for i, (status, res, lat) in zip(order, done):
        assert status == relo.OK and lat > 0
        assert res.as_dict() == alone[i]
    ctx.close()


def test_served_admission_by_budget(relo, workload):
    ctx, reqs = served_setup(relo, workload)
    alone = [ctx.relocalize(*r).as_dict() for r in reqs]
    ctx.serve_start(max_batch=8, max_inflight=2, hbm_budget=1024)      # smaller than any request's scratch
    t = ctx.submit(*reqs[1])
    (status, res, lat), = poll_all(ctx, [t])
    assert status == relo.E_OVER_BUDGET
    ctx.serve_stop()
    ctx.serve_start(max_batch=8, max_inflight=2, hbm_budget=8 << 20)   # room for a request or two at a time
    tickets = [ctx.submit(*r) for r in reqs]
    done = poll_all(ctx, tickets)
    ctx.serve_stop()
    for i, (status, res, lat) in enumerate(done):
        assert status == relo.OK and res.as_dict() == alone[i]
    ctx.close()


def test_served_request_deadlines(relo, workload):
    """A served request whose deadline passes while it waits for admission
    completes with RELO_E_TIMEOUT and is never launched; the others run as
    alone.  One slot and one request per batch: the second request can only be
    admitted once the first has left the GPU, long after its 1-microsecond
    deadline; the third has a deadline it can meet."""
    ctx, reqs = served_setup(relo, workload)
    alone = [ctx.relocalize(*r).as_dict() for r in reqs]
    ctx.serve_start(max_batch=1, max_inflight=1)
    t_first = ctx.submit(*reqs[0])
    t_late = ctx.submit(*reqs[1], timeout_s=1e-6)
    t_ok = ctx.submit(*reqs[2], timeout_s=60.0)
    first, late, ok = poll_all(ctx, [t_first, t_late, t_ok])
    ctx.serve_stop()
    assert first[0] == relo.OK and first[1].as_dict() == alone[0]
    assert late[0] == relo.E_TIMEOUT
    assert ok[0] == relo.OK and ok[1].as_dict() == alone[2]
    with pytest.raises(relo.ReloError):
        ctx.serve_start(max_batch=1, max_inflight=1)
        try:
            ctx.submit(*reqs[0], timeout_s=-1.0)
        finally:
            ctx.serve_stop()
    ctx.close()


def test_map_update_then_relocalize_without_waiting(relo, workload):
    """relo_update_map_dev runs the field part of the EDT on a second stream,
    overlapping the next request's ray cast; TAM and the table export wait for
    it.  Back-to-back updates between two maps, each followed at once by a
    relocalization and by the exported d2, give what a fresh context with
    that map gives, and d2 equals the oracle's EDT."""
    torch = torch_()
    wl = workload(1)
    other = workloads.make_office(77)
    hyps = wl.hyps[other[wl.hyps[:, 1], wl.hyps[:, 0]] < 65]   # free on both maps
    ref = {}
    for name, g in (("a", wl.grid), ("b", other)):
        c = relo.Relo(n_orient=wl.n_orient, topk=64, early_stop=0)
        m = c.load_map(g, wl.res)
        c.set_hypotheses(m, workloads.cell_centres(hyps, wl.res))
        ref[name] = c.relocalize(m, wl.ranges, wl.angles, wl.max_range).as_dict()
        c.close()
    ctx = relo.Relo(n_orient=wl.n_orient, topk=64, early_stop=0)
    mid = ctx.load_map(wl.grid, wl.res)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, wl.res))
    grids = {"a": torch.tensor(wl.grid, device="cuda"), "b": torch.tensor(other, device="cuda")}
    z = torch.tensor(wl.ranges, device="cuda")
    out = torch.empty(relo.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for name in ("b", "a", "b", "b", "a"):
        ctx.update_map_dev(mid, grids[name])
        ctx.relocalize_dev(mid, z, wl.angles, wl.max_range, out)
        got = relo.result_from_bytes(bytes(out.cpu().numpy())).as_dict()
        assert got == ref[name], name
    ctx.update_map_dev(mid, grids["b"])
    d2, _, _ = ctx.map_tables(mid, other.shape)
    assert np.array_equal(d2.cpu().numpy().astype(np.int64), oracle.edt(other))
    ctx.close()


def test_launch_shapes_do_not_change_results(relo, workload):
    """The autotuner's knobs (survivors per TAM task, resident CTAs per SM of
    TAM and of the ray cast) change only the time: every TAM score and the
    result are bitwise those of the built-in shapes; malformed entries are
    rejected."""
    torch = torch_()
    wl = workload(1)
    K = wl.topk
    ctx = relo.Relo(n_orient=wl.n_orient, topk=K, early_stop=0)
    mid = ctx.load_map(wl.grid, wl.res)
    ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))

    def scores():
        r = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range).as_dict()
        T = ctx.stage(relo.STAGE_TAM, torch.empty(K * wl.n_orient, dtype=torch.float32, device="cuda"))
        return r, T.cpu().numpy()
    base, T0 = scores()
    cls = relo.tam_class(len(wl.ranges))
    for entries in ([(relo.TUNE_TAM, (cls, wl.n_orient, K), (8, 1))],
                    [(relo.TUNE_TAM, (0, 0, 0), (64, 2)), (relo.TUNE_CAST, (0, 0, 0), (2, 0))],
                    [(relo.TUNE_TAM, (cls, 0, 0), (128, 0)), (relo.TUNE_CAST, (wl.n_s, 0, 0), (1, 0))],
                    # a single request's own entry comes first, the batched one is the fallback
                    [(relo.TUNE_TAM_ONE, (cls, wl.n_orient, K), (16, 3)), (relo.TUNE_TAM, (0, 0, 0), (8, 1))]):
        ctx.set_tuning(entries)
        got, T = scores()
        assert got == base
        assert np.array_equal(T.view(np.uint32), T0.view(np.uint32))
    for bad in ([(relo.TUNE_TAM, (0, 0, 0), (12, 0))], [(9, (0, 0, 0), (8, 0))], [(relo.TUNE_CAST, (0, 0, 0), (-1, 0))],
                [(relo.TUNE_TAM_ONE, (0, 0, 0), (136, 0))]):
        with pytest.raises(relo.ReloError):
            ctx.set_tuning(bad)
    ctx.set_tuning([])
    ctx.close()


def test_survivors_when_every_smad_ties(relo):
    """A map without obstacles: every synthesized scan is empty, every SMAD
    numerator is the same, and the survivor keys differ only in the hypothesis
    index.  The top-K's first 11-bit histogram then puts every key in one bin
    (the radix-select path); the survivors must be the K lowest indices."""
    torch = torch_()
    g = np.zeros((80, 96), np.int8)
    rng = np.random.default_rng(12)
    cells = np.stack([rng.integers(0, 96, 300), rng.integers(0, 80, 300)], 1).astype(np.int32)
    cells = np.unique(cells, axis=0)
    ang = workloads.beam_angles(90, 120)
    z = np.full(90, 3.0, np.float32)
    for K in (16, 100):
        ctx = relo.Relo(n_orient=40, topk=K, batch=K, local_topk=4, early_stop=0, max_range=5.0)
        mid = ctx.load_map(g, 0.05)
        ctx.set_hypotheses(mid, workloads.cell_centres(cells, 0.05))
        res = ctx.relocalize(mid, z, ang, 4.0)
        assert res.status == relo.OK
        num = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(cells), dtype=torch.int64, device="cuda")).cpu().numpy()
        surv = ctx.stage(relo.STAGE_SURVIVORS, torch.empty(K, dtype=torch.int32, device="cuda")).cpu().numpy()
        assert (num == num[0]).all()
        assert np.array_equal(surv, np.arange(K))
        assert np.array_equal(surv, oracle.rank(num, K))
        ctx.close()
