"""The two ray traversals (Eq. 13): per-direction tables (tile by tile) and
cell-by-cell stepping give the same cells, hits and ranges, which are the
oracle's.

The tables are built once per (N_s, range limit) from the integer DDA of
every direction; the tile walk then moves tile to tile and finds the first
occupied cell with a bit board.  Maps whose sides are not multiples of the
8-cell tile, hypotheses next to the border, short and long range limits,
axis-aligned directions and open maps whose rays leave whole empty squares of
tiles at once are covered, against the oracle's exact traversal.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


def synth(relo, grid, cells, angles, scan_range, ns, **params):
    import torch
    ctx = relo.Relo(**params)
    mid = ctx.load_map(grid, 0.05)
    c = torch.tensor(cells, dtype=torch.int32, device="cuda")
    r, h = ctx.synth_scans(mid, c, angles, scan_range, ns)
    ctx.close()
    return r.cpu().numpy().view(np.uint32).astype(np.int64), h.cpu().numpy()


@pytest.mark.parametrize("shape,density,max_range,n_beams,ns", [
    ((197, 203), 0.0, 6.0, 120, 120),       # office cut to odd sides, panoramic (the four axis directions included)
    ((61, 45), 0.04, 3.0, 64, 96),          # random obstacles, short range
    ((64, 64), 0.002, 30.0, 72, 72),        # nearly empty: rays leave the map
    ((130, 9), 0.01, 2.0, 50, 100),         # thin map, range limit inside the first tiles
    ((300, 517), 0.0003, 20.0, 180, 360),   # open map: rays leave whole empty squares of tiles, up to the border
    ((601, 587), -1.0, 25.0, 360, 720),     # warehouse rows: long rays down the aisles through empty squares
])
def test_tables_equal_stepping_and_oracle(relo, shape, density, max_range, n_beams, ns):
    rng = np.random.default_rng(hash(shape) % 1000)
    H, W = shape
    if density == 0.0:
        g = workloads.make_office(3, n=max(H, W) + 8)[:H, :W].copy()
    elif density < 0.0:
        g = workloads.make_warehouse(5, n=max(H, W) + 8)[:H, :W].copy()
    else:
        g = np.where(rng.random(shape) < density, 100, 0).astype(np.int8)
    free = np.argwhere(g < 65)[:, ::-1]
    pick = free[rng.choice(len(free), 40, replace=False)]
    border = np.array([[0, 0], [W - 1, H - 1], [0, H - 1], [W - 1, 0]])
    border = border[[g[y, x] < 65 for x, y in border]]
    cells = np.concatenate([pick, border]).astype(np.int32)
    ang = workloads.beam_angles(n_beams, ns)
    prm = dict(n_orient=0, max_range=max_range + 1.0)
    r1, h1 = synth(relo, g, cells, ang, max_range, ns, ray_tables=1, **prm)
    r0, h0 = synth(relo, g, cells, ang, max_range, ns, ray_tables=0, **prm)
    assert np.array_equal(r1, r0) and np.array_equal(h1, h0)
    pl = oracle.plan(np.full(n_beams, max_range * 0.5, np.float32), ang, max_range, 0.05,
                     oracle.Params(n_orient=0))
    assert pl["ns"] == ns
    for k, (x, y) in enumerate(cells):
        want_r, hx, hy = oracle.synth_scan(g, int(x), int(y), pl)
        assert np.array_equal(r1[k], want_r)
        assert np.array_equal(h1[k], np.where(hx < 0, -1, hy * W + hx))


def walk_boxes_definition(g):
    """The empty boxes of every walk-frame tile, from their definition by 2-D
    prefix counts of non-empty tiles (see relo_map_walk_boxes_dev)."""
    H, W = g.shape
    TW, TH = (W + 7) // 8, (H + 7) // 8
    occ = np.ones((TH * 8, TW * 8), bool)
    occ[:H, :W] = g >= 65
    ne = occ.reshape(TH, 8, TW, 8).any(axis=(1, 3))
    out = np.zeros((4, TH + 1, TW + 1), np.int64)
    y = np.arange(TH + 1)[:, None]
    x = np.arange(TW + 1)[None, :]
    for f in range(4):
        t = ne[:, ::-1] if f & 1 else ne
        t = t[::-1, :] if f & 2 else t
        full = np.ones((TH + 1 + 16, TW + 1 + 16), np.int64)   # the border row and column, and beyond, count as full
        full[:TH, :TW] = t
        c = np.zeros((full.shape[0] + 1, full.shape[1] + 1), np.int64)
        c[1:, 1:] = full.cumsum(0).cumsum(1)

        def empty(h, w):   # every tile of [x, x + w) x [y, y + h) empty
            return (c[y + h, x + w] - c[y, x + w] - c[y + h, x] + c[y, x]) == 0
        s = sum(empty(k, k).astype(np.int64) for k in range(1, 17))
        xr = sum(empty(1, k).astype(np.int64) for k in range(1, 17))
        yr = sum(empty(k, 1).astype(np.int64) for k in range(1, 17))
        out[f] = s | (xr << 5) | (yr << 10)
    return out


@pytest.mark.parametrize("shape,density", [
    ((1000, 1000), 0.0),      # all free: rows of more than 64 empty tiles, whole squares of 16
    ((300, 517), 0.0003),     # nearly empty, sides not multiples of 8
    ((601, 587), -1.0),       # warehouse rows
    ((1, 1), 0.0), ((9, 17), 0.0), ((130, 9), 0.01), ((257, 263), 0.002),
])
def test_walk_boxes_match_definition(relo, shape, density):
    rng = np.random.default_rng(7)
    H, W = shape
    if density < 0.0:
        g = workloads.make_warehouse(5, n=max(H, W) + 8)[:H, :W].copy()
    else:
        g = np.where(rng.random(shape) < density, 100, 0).astype(np.int8)
    ctx = relo.Relo(n_orient=0)
    mid = ctx.load_map(g, 0.05)
    got = ctx.walk_boxes(mid, g.shape)
    # after an update the boxes follow the new grid
    g2 = g.copy()
    g2[H // 2, :] = 100
    ctx.update_map(mid, g2)
    got2 = ctx.walk_boxes(mid, g2.shape)
    ctx.close()
    assert np.array_equal(got, walk_boxes_definition(g))
    assert np.array_equal(got2, walk_boxes_definition(g2))


@pytest.mark.parametrize("cfg", [0, 1])
def test_full_path_same_with_either_traversal(relo, workload, cfg):
    wl = workload(cfg)
    K = 16 if cfg == 0 else 256
    out = []
    for rt in (1, 0):
        ctx = relo.Relo(n_orient=wl.n_orient, topk=K, early_stop=0, ray_tables=rt)
        mid = ctx.load_map(wl.grid, wl.res)
        ctx.set_hypotheses(mid, workloads.cell_centres(wl.hyps, wl.res))
        res = ctx.relocalize(mid, wl.ranges, wl.angles, wl.max_range).as_dict()
        import torch
        num = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(wl.hyps), dtype=torch.int64, device="cuda")).cpu()
        out.append((res, num.numpy()))
        ctx.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
