"""Positional hypotheses by the traversability-constrained RRT (Algorithm 1)
on the GPU.

The GPU sampler searches the nearest nodes of a sub-batch of points at once
and then resolves the sub-batch in sample order, so it must grow exactly the
tree that Algorithm 1 grows one point at a time from the same random points
in float32: the representatives, the rounds and the tree size are compared
bit for bit with the serial float32 program (tests/rrt_f32.py).  Against the
serial generator that builds the workloads' hypotheses (other random points),
what must agree is what the hypotheses are for (Sec. III-A): the reachable
free space is covered as well (every traversable cell reachable from the
start lies within one voxel diagonal of a hypothesis as often), about as many
hypotheses come out, each on a traversable cell, at most one per voxel of
side rho, and a seed gives the same set every time.
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RES = 0.05
R_ROBOT = 0.21


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


def coverage(xy, clr, p0, radius):
    """Fraction of the traversable cells reachable from p0 (4-connected) within radius of a hypothesis."""
    from scipy.ndimage import label
    from scipy.spatial import cKDTree
    lab, _ = label(clr >= R_ROBOT)
    reach = lab == lab[int(p0[1] / RES), int(p0[0] / RES)]
    ys, xs = np.nonzero(reach)
    d, _ = cKDTree(xy).query(np.stack([(xs + 0.5) * RES, (ys + 0.5) * RES], 1))
    return float((d <= radius).mean())


def scene(which):
    g = {"room": lambda: workloads.make_room(1000),
         "office": lambda: workloads.make_office(1001)[:256, :256],
         "office512": lambda: workloads.make_office(1001)[:512, :512]}[which]()
    clr = workloads.clearance_table(g, RES)
    p0 = workloads.free_start(g, RES, R_ROBOT, 7, clr)
    n_target = {"room": 200, "office": 600, "office512": 2000}[which]
    rho = math.sqrt(float((clr >= R_ROBOT).sum()) * RES * RES / (1.1 * n_target))
    return g, clr, p0, rho


@pytest.mark.parametrize("which,seed", [("room", 7), ("room", 123), ("office", 7), ("office512", 7)])
def test_gpu_rrt_is_the_serial_tree(relo, which, seed):
    import torch
    from rrt_f32 import serial_rrt
    g, clr, p0, rho = scene(which)
    want, want_rounds, want_nodes = serial_rrt(clr, RES, p0, rho, 0.6, R_ROBOT, 2, seed)
    ctx = relo.Relo()
    xy_d, rounds, nodes = ctx.rrt_hypotheses(torch.tensor(clr, device="cuda"), RES, p0, rho, 0.6, R_ROBOT, 2,
                                             seed=seed)
    ctx.close()
    assert (rounds, nodes) == (want_rounds, want_nodes)
    assert np.array_equal(xy_d.cpu().numpy(), want)


def test_gpu_rrt_node_cap_ends_the_tree_like_the_serial_program(relo):
    import torch
    from rrt_f32 import serial_rrt
    g, clr, p0, rho = scene("room")
    want, want_rounds, want_nodes = serial_rrt(clr, RES, p0, rho, 0.6, R_ROBOT, 2, 7, node_cap=300)
    ctx = relo.Relo()
    xy_d, rounds, nodes = ctx.rrt_hypotheses(torch.tensor(clr, device="cuda"), RES, p0, rho, 0.6, R_ROBOT, 2,
                                             seed=7, node_cap=300)
    ctx.close()
    assert nodes == want_nodes == 300 and rounds == want_rounds
    assert np.array_equal(xy_d.cpu().numpy(), want)


@pytest.mark.parametrize("which", ["room", "office"])
def test_gpu_rrt_covers_like_the_serial_sampler(relo, which):
    import torch
    g, clr, p0, rho = scene(which)
    xs, _, _ = workloads.rrt(g, RES, p0, rho, 0.6, R_ROBOT, 2, 7, clr=clr)
    ctx = relo.Relo()
    clr_d = torch.tensor(clr, device="cuda")
    xy_d, rounds, nodes = ctx.rrt_hypotheses(clr_d, RES, p0, rho, 0.6, R_ROBOT, 2, seed=7)
    xy = xy_d.cpu().numpy()
    again, _, _ = ctx.rrt_hypotheses(clr_d, RES, p0, rho, 0.6, R_ROBOT, 2, seed=7)
    ctx.close()
    assert np.array_equal(again.cpu().numpy(), xy)                     # deterministic for a seed
    assert 0.8 * len(xs) <= len(xy) <= 1.25 * len(xs)
    radius = rho * math.sqrt(2.0)
    assert coverage(xy.astype(np.float64), clr, p0, radius) >= coverage(xs, clr, p0, radius) - 0.02
    cells = np.floor(xy / np.float32(RES)).astype(np.int64)             # the kernel's float32 cell rule
    c = clr[cells[:, 1], cells[:, 0]]
    assert (c >= R_ROBOT - RES).all() and (c >= R_ROBOT).mean() >= 0.99
    vox = np.floor(xy.astype(np.float64) / rho).astype(np.int64)
    assert len(np.unique(vox, axis=0)) >= 0.99 * len(vox)               # one per voxel (float32 edges aside)
    assert np.allclose(xy[0], p0, atol=1e-5) and rounds >= 2 and nodes >= len(xy)


def test_gpu_rrt_rejects_a_start_off_the_map(relo):
    import torch
    g, clr, p0, rho = scene("room")
    ctx = relo.Relo()
    with pytest.raises(relo.ReloError):
        ctx.rrt_hypotheses(torch.tensor(clr, device="cuda"), RES, (-1.0, 0.5), rho)
    ctx.close()


def blocked_clearance(g):
    """MinDistToObstacle by definition, from the oracle's exact EDT: the grid
    with a ring of blocked cells around it, every cell blocked that is
    occupied (>= 65) or unknown (< 0); clearance = res * sqrt(d2) in FP64,
    rounded once to float32."""
    import oracle
    ring = np.full((g.shape[0] + 2, g.shape[1] + 2), 100, np.int8)
    ring[1:-1, 1:-1] = np.where((g < 0) | (g >= 65), 100, 0)
    d2 = oracle.edt(ring)[1:-1, 1:-1]
    return (RES * np.sqrt(d2.astype(np.float64))).astype(np.float32)


@pytest.mark.parametrize("which", ["room", "office512"])
def test_rrt_from_the_grid(relo, which):
    """relo_rrt_sample builds the clearance table from the grid with the
    library's EDT (bit for bit the definition over the oracle's EDT, and the
    table the workloads computed with SciPy), then grows the same tree as the
    clearance-taking sampler."""
    import torch
    g, clr, p0, rho = scene(which)
    ctx = relo.Relo()
    xy, rounds, nodes, got_clr = ctx.rrt_sample(g, RES, p0, rho, 0.6, R_ROBOT, 2, seed=11, with_clearance=True)
    assert np.array_equal(got_clr, blocked_clearance(g))
    assert np.array_equal(got_clr, clr)
    ref, r_ref, n_ref = ctx.rrt_hypotheses(torch.tensor(clr, device="cuda"), RES, p0, rho, 0.6, R_ROBOT, 2, seed=11)
    ctx.close()
    assert (rounds, nodes) == (r_ref, n_ref)
    assert np.array_equal(xy, ref.cpu().numpy().astype(np.float64))
    assert len(xy) > 0


def test_rrt_from_the_grid_rejects_a_start_off_the_map(relo):
    g = workloads.make_room(1000)
    ctx = relo.Relo()
    with pytest.raises(relo.ReloError) as e:
        ctx.rrt_sample(g, RES, (-1.0, 0.5), 0.3)
    assert e.value.code == relo.E_INVALID_ARG
    ctx.close()
