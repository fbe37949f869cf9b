"""Resident synthesized scans: reading a stored table gives the same results as casting.

The synthesized panoramic scan of a hypothesis (Eq. 13) depends on the map,
the hypothesis, N_s and the range limit only, so a table stored by one
request and read by a later one must reproduce every integer stage output
bit for bit and every TAM score exactly (the same arithmetic runs on the same
ranges).  The path that casts is itself checked against the oracle in
test_gpu_parity.py; here every comparison is against a context without the
cache.  Also covered: invalidation when the map or the hypotheses change,
LRU eviction under a small budget, two requests of one geometry in one batch,
a batch mixing a request that reads stored scans with one that casts, and the
served form.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

GIB = 1 << 30


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


def stage_arrays(relo, ctx, n_hyp, K, n_orient):
    import torch
    out = {}
    for name, which, n, dt in (("num", relo.STAGE_SMAD_NUM, n_hyp, torch.int64),
                               ("m", relo.STAGE_SMAD_M, n_hyp, torch.int32),
                               ("surv", relo.STAGE_SURVIVORS, K, torch.int32),
                               ("T", relo.STAGE_TAM, K * n_orient, torch.float32),
                               ("best_m", relo.STAGE_BEST_M, K, torch.int32)):
        out[name] = ctx.stage(which, torch.empty(n, dtype=dt, device="cuda")).cpu().numpy()
    out["T"] = out["T"].view(np.uint32)   # bitwise, NaN (unscored) included
    return out


def assert_same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def fresh_result(relo, grid, res, hyps, z, ang, mr, **params):
    ctx = relo.Relo(**params)
    mid = ctx.load_map(grid, res)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, res))
    out = ctx.relocalize(mid, z, ang, mr).as_dict()
    ctx.close()
    return out


def test_office_table_read_equals_cast(relo, workload):
    wl = workload(1)
    K, n_orient = 256, wl.n_orient
    plain = relo.Relo(n_orient=n_orient, topk=K, early_stop=0)
    cached = relo.Relo(n_orient=n_orient, topk=K, early_stop=0, scan_cache_bytes=GIB)
    ids = []
    for ctx in (plain, cached):
        mid = ctx.load_map(wl.grid, wl.res)
        ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
        ids.append(mid)
    want = plain.relocalize(ids[0], wl.ranges, wl.angles, wl.max_range).as_dict()
    want_st = stage_arrays(relo, plain, len(wl.hyps), K, n_orient)
    for rep in range(3):
        # call 0 casts, stores the ranges and builds the window table; calls 1 and 2 read the windows
        got = cached.relocalize(ids[1], wl.ranges, wl.angles, wl.max_range).as_dict()
        assert got == want
        assert_same(stage_arrays(relo, cached, len(wl.hyps), K, n_orient), want_st)
        st = cached.scan_cache_stats()
        assert st["tables"] == 1 and st["misses"] == 1 and st["hits"] == rep
        assert st["win_tables"] == 1 and st["win_hits"] == rep
        assert st["bytes"] == 4 * len(wl.hyps) * 1440 + 8 * len(wl.hyps) * n_orient
        info = cached.scan_info()
        assert (info[8] == 0) == (rep > 0)   # no ray is cast once the table is stored
    plain.close()
    cached.close()


def small_map(seed=5, n=128, n_hyp=400):
    g = workloads.make_office(seed, n=n)
    free = np.argwhere(g == 0)[:, ::-1]
    hyps = free[np.random.default_rng(seed).choice(len(free), n_hyp, replace=False)].astype(np.int32)
    return g, hyps


def scan_from(g, hyps, idx, n_beams, ns, theta, mr=4.0, seed=0):
    ang = workloads.beam_angles(n_beams, ns)
    h = hyps[idx]
    z = workloads.render_scan(g, 0.05, ((h[0] + 0.5) * 0.05, (h[1] + 0.5) * 0.05, theta), ang, mr)
    return workloads.add_noise(z, mr, seed), ang


def test_tables_dropped_on_map_and_hypothesis_change(relo):
    g, hyps = small_map()
    z, ang = scan_from(g, hyps, 17, 90, 120, 0.4)
    prm = dict(n_orient=40, topk=24, batch=8, local_topk=4, early_stop=0, max_range=5.0)
    ctx = relo.Relo(scan_cache_bytes=GIB, **prm)
    mid = ctx.load_map(g, 0.05)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == fresh_result(relo, g, 0.05, hyps, z, ang, 4.0, **prm)
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == fresh_result(relo, g, 0.05, hyps, z, ang, 4.0, **prm)
    assert ctx.scan_cache_stats()["hits"] == 1
    # a new obstacle changes the synthesized scans: the stored table must not be read
    g2 = g.copy()
    free = np.argwhere(g2 == 0)
    occupied = set()
    for (y, x) in free[np.random.default_rng(1).choice(len(free), 300, replace=False)]:
        g2[y, x] = 100
        occupied.add((x, y))
    keep = np.array([(int(h[0]), int(h[1])) not in occupied for h in hyps])
    ctx.update_map(mid, g2)
    assert ctx.scan_cache_stats()["tables"] == 0
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps[keep], 0.05))
    want = fresh_result(relo, g2, 0.05, hyps[keep], z, ang, 4.0, **prm)
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    # another hypothesis set on the same map
    sub = hyps[keep][::3]
    ctx.set_hypotheses(mid, workloads.cell_centres(sub, 0.05))
    assert ctx.scan_cache_stats()["tables"] == 0
    want = fresh_result(relo, g2, 0.05, sub, z, ang, 4.0, **prm)
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    st = ctx.scan_cache_stats()
    assert st["hits"] == 3 and st["misses"] == 3
    ctx.close()


def test_small_budget_evicts_least_recently_used(relo):
    g, hyps = small_map(seed=6)
    za, anga = scan_from(g, hyps, 3, 90, 120, 1.0, seed=1)     # N_s 120: 192000-byte table
    zb, angb = scan_from(g, hyps, 9, 100, 160, -2.0, seed=2)   # N_s 160: 256000-byte table
    prm = dict(n_orient=40, topk=16, batch=8, local_topk=4, early_stop=1, tau=0.9, max_range=5.0)
    want_a = fresh_result(relo, g, 0.05, hyps, za, anga, 4.0, **prm)
    want_b = fresh_result(relo, g, 0.05, hyps, zb, angb, 4.0, **prm)
    ctx = relo.Relo(scan_cache_bytes=300000, **prm)
    mid = ctx.load_map(g, 0.05)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
    for which in "ababaa":
        z, ang, want = (za, anga, want_a) if which == "a" else (zb, angb, want_b)
        assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    st = ctx.scan_cache_stats()
    # a window table (400 x 40 x 8 B) never fits beside its scan table in this budget
    assert st == {"tables": 1, "bytes": 192000, "hits": 1, "misses": 5, "evictions": 4, "win_tables": 0,
                  "win_hits": 0}
    ctx.close()
    # a table larger than the whole budget is never stored
    ctx = relo.Relo(scan_cache_bytes=1000, **prm)
    mid = ctx.load_map(g, 0.05)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
    for _ in range(2):
        assert ctx.relocalize(mid, za, anga, 4.0).as_dict() == want_a
    assert ctx.scan_cache_stats() == {"tables": 0, "bytes": 0, "hits": 0, "misses": 2, "evictions": 0,
                                      "win_tables": 0, "win_hits": 0}
    ctx.close()


def test_one_geometry_twice_in_one_batch(relo):
    g, hyps = small_map(seed=7)
    z1, ang = scan_from(g, hyps, 5, 90, 120, 0.3, seed=3)
    z2, _ = scan_from(g, hyps, 50, 90, 120, 2.5, seed=4)
    prm = dict(n_orient=40, topk=16, batch=8, local_topk=4, early_stop=0, max_range=5.0)
    want = [fresh_result(relo, g, 0.05, hyps, z, ang, 4.0, **prm) for z in (z1, z2)]
    ctx = relo.Relo(scan_cache_bytes=GIB, **prm)
    mid = ctx.load_map(g, 0.05)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
    items = [(mid, z1, ang, 4.0), (mid, z2, ang, 4.0)]
    # first batch: request 0 stores the table and builds its window table, request 1 casts into its
    # scratch; second batch: both read the window table
    for _ in range(2):
        assert [r.as_dict() for r in ctx.relocalize_batch(items)] == want
    assert ctx.scan_cache_stats() == {"tables": 1, "bytes": 4 * len(hyps) * 120 + 8 * len(hyps) * 40, "hits": 2,
                                      "misses": 2, "evictions": 0, "win_tables": 1, "win_hits": 2}
    ctx.close()


@pytest.mark.parametrize("reader_first", [True, False])
def test_batch_mixing_stored_and_cast_scans(relo, reader_first):
    """One batch in which one request reads its map's resident scans and the
    other casts rays: the ray-cast launch prepares both requests' real scans
    (Eq. 16, 26-27), the reader's included, whichever place it takes."""
    g1, h1 = small_map(seed=8)
    g2, h2 = small_map(seed=9, n=96, n_hyp=300)
    z1, ang = scan_from(g1, h1, 3, 90, 120, 0.7, seed=5)
    z2, _ = scan_from(g2, h2, 9, 90, 120, -1.1, seed=6)
    prm = dict(n_orient=40, topk=16, batch=8, local_topk=4, early_stop=0, max_range=5.0)
    want1 = fresh_result(relo, g1, 0.05, h1, z1, ang, 4.0, **prm)
    want2 = fresh_result(relo, g2, 0.05, h2, z2, ang, 4.0, **prm)
    ctx = relo.Relo(scan_cache_bytes=GIB, **prm)
    m1 = ctx.load_map(g1, 0.05)
    ctx.set_hypotheses(m1, workloads.cell_centres(h1, 0.05))
    m2 = ctx.load_map(g2, 0.05)
    ctx.set_hypotheses(m2, workloads.cell_centres(h2, 0.05))
    assert ctx.relocalize(m1, z1, ang, 4.0).as_dict() == want1   # stores map 1's scans
    items = [(m1, z1, ang, 4.0), (m2, z2, ang, 4.0)]
    want = [want1, want2]
    if not reader_first:
        items, want = items[::-1], want[::-1]
    assert [r.as_dict() for r in ctx.relocalize_batch(items)] == want
    st = ctx.scan_cache_stats()
    assert st["tables"] == 2 and st["misses"] == 2 and st["hits"] == 1
    ctx.close()


def test_caer_reads_stored_scans_without_window_tables(relo):
    """CAER needs the synthesized rows themselves: with resident scans it reads
    the stored table and builds no window table (those serve SMAD only)."""
    g, hyps = small_map(seed=10)
    z, ang = scan_from(g, hyps, 12, 90, 120, 1.9, seed=7)
    prm = dict(n_orient=40, topk=16, batch=8, local_topk=4, early_stop=0, max_range=5.0, coarse_metric=1)
    want = fresh_result(relo, g, 0.05, hyps, z, ang, 4.0, **prm)
    ctx = relo.Relo(scan_cache_bytes=GIB, **prm)
    mid = ctx.load_map(g, 0.05)
    ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
    for _ in range(3):
        assert ctx.relocalize(mid, z, ang, 4.0).as_dict() == want
    st = ctx.scan_cache_stats()
    assert st["tables"] == 1 and st["hits"] == 2 and st["misses"] == 1
    assert st["win_tables"] == 0 and st["win_hits"] == 0
    ctx.close()


def test_served_stream_with_tables_equals_alone(relo):
    """Served form with resident scans: requests on several maps and sensors,
    in waves while others run, each give their alone (uncached) result."""
    prm = dict(n_orient=40, topk=16, batch=8, local_topk=4, early_stop=1, tau=0.9, max_range=5.0)
    plain = relo.Relo(**prm)
    served = relo.Relo(scan_cache_bytes=GIB, **prm)
    reqs_plain, reqs_served = [], []
    for seed in (11, 12):
        g, hyps = small_map(seed=seed, n=96 + 32 * (seed - 11), n_hyp=300 + 100 * (seed - 11))
        for ctx, reqs in ((plain, reqs_plain), (served, reqs_served)):
            mid = ctx.load_map(g, 0.05)
            ctx.set_hypotheses(mid, workloads.cell_centres(hyps, 0.05))
            for k, (nb, ns) in enumerate(((90, 120), (100, 160), (120, 120))):
                z, ang = scan_from(g, hyps, 7 * k + seed, nb, ns, 0.5 * k - 1.0, seed=seed + k)
                reqs.append((mid, z, ang, 4.0))
    alone = [plain.relocalize(*r).as_dict() for r in reqs_plain]
    served.serve_start(max_batch=3, max_inflight=2)
    order = [(5 * i) % len(reqs_served) for i in range(24)]
    tickets = [served.submit(*reqs_served[i]) for i in order[:10]]
    tickets += [served.submit(*reqs_served[i]) for i in order[10:]]
    import time
    got, t0 = {}, time.time()
    while len(got) < len(tickets):
        for t in tickets:
            if t not in got:
                r = served.poll(t)
                if r is not None:
                    got[t] = r
        assert time.time() - t0 < 60.0
        time.sleep(0.001)
    served.serve_stop()
    for i, t in zip(order, tickets):
        status, res, lat = got[t]
        assert status == relo.OK and res.as_dict() == alone[i]
    st = served.scan_cache_stats()
    assert st["tables"] == 4 and st["hits"] > 0 and st["hits"] + st["misses"] == len(tickets)
    assert st["win_tables"] == 6 and st["win_hits"] > 0   # three plans per map, two sharing N_s = 120
    plain.close()
    served.close()


def test_window_search_keeps_the_smaller_m_on_ties(relo):
    """A square room seen from points on its axes of symmetry: many orientations
    give the same window sum, and pairs of orientations lie at the same distance
    on either side of sum R_real.  SMAD by window search must pick the same
    (numerator, m) as the direct minimum, smaller m on every tie."""
    import torch
    n = 96
    g = np.zeros((n, n), np.int8)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 100
    c = n // 2
    cells = np.array([[c, c], [c, c - 20], [c - 20, c], [c + 13, c + 13], [c - 7, c + 7], [c, 9]], np.int32)
    prm = dict(n_orient=40, topk=6, batch=6, local_topk=3, early_stop=0, max_range=6.0)
    for n_beams, ns, theta in ((90, 120, 0.0), (60, 120, np.pi / 2), (100, 160, 0.3)):
        ang = workloads.beam_angles(n_beams, ns)
        for h in range(len(cells)):
            z = workloads.render_scan(g, 0.05, ((cells[h, 0] + 0.5) * 0.05, (cells[h, 1] + 0.5) * 0.05, theta), ang, 5.0)
            out = []
            for cache in (0, GIB):
                ctx = relo.Relo(scan_cache_bytes=cache, **prm)
                mid = ctx.load_map(g, 0.05)
                ctx.set_hypotheses(mid, workloads.cell_centres(cells, 0.05))
                for _ in range(2 if cache else 1):   # with the cache, the second call reads the window table
                    res = ctx.relocalize(mid, z, ang, 5.0).as_dict()
                num = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(cells), dtype=torch.int64, device="cuda")).cpu()
                mm = ctx.stage(relo.STAGE_SMAD_M, torch.empty(len(cells), dtype=torch.int32, device="cuda")).cpu()
                if cache:
                    assert ctx.scan_cache_stats()["win_hits"] == 1
                out.append((res, num.numpy(), mm.numpy()))
                ctx.close()
            assert out[0][0] == out[1][0]
            assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
