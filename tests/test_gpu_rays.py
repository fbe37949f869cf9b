"""The two ray traversals (Eq. 13): per-direction tables (tile by tile) and
cell-by-cell stepping give the same cells, hits and ranges, which are the
oracle's.

The tables are built once per (N_s, range limit) from the integer DDA of
every direction; the tile walk then moves tile to tile and finds the first
occupied cell with a bit board.  Maps whose sides are not multiples of the
8-cell tile, hypotheses next to the border, short and long range limits and
axis-aligned directions are covered, against the oracle's exact traversal.
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
])
def test_tables_equal_stepping_and_oracle(relo, shape, density, max_range, n_beams, ns):
    rng = np.random.default_rng(hash(shape) % 1000)
    H, W = shape
    if density == 0.0:
        g = workloads.make_office(3, n=max(H, W) + 8)[:H, :W].copy()
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
