"""The serial float32 program of Algorithm 1 (tests/rrt_f32.py) that the GPU
sampler must reproduce bit for bit, pinned on the CPU: its generator against
the published SplitMix64 stream, and its trees against the independent serial
generator that builds the workloads' hypotheses (other random points, float64
positions): as many hypotheses, the same coverage of the reachable free space,
every representative traversable and alone in its voxel."""
import math

import numpy as np
import pytest

import workloads
from rrt_f32 import serial_rrt, splitmix64, unit_draw

RES = 0.05
R_ROBOT = 0.21


def test_splitmix64_matches_the_published_stream():
    # SplitMix64 seeded with 0: the state advances by the golden gamma before each output
    gamma = 0x9E3779B97F4A7C15
    outs = [splitmix64((k * gamma) & ((1 << 64) - 1)) for k in range(3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_unit_draws_are_float32_in_the_unit_interval_and_keyed():
    d = np.array([unit_draw(5, r, i, k) for r in range(3) for i in range(200) for k in range(2)])
    assert d.dtype == np.float32 and (d >= 0).all() and (d < 1).all()
    assert abs(float(d.mean()) - 0.5) < 0.03
    assert len(np.unique(d)) == len(d)
    assert unit_draw(5, 1, 2, 0) != unit_draw(6, 1, 2, 0) != unit_draw(5, 1, 2, 1)


def coverage(xy, clr, p0, radius):
    from scipy.ndimage import label
    from scipy.spatial import cKDTree
    lab, _ = label(clr >= R_ROBOT)
    reach = lab == lab[int(p0[1] / RES), int(p0[0] / RES)]
    ys, xs = np.nonzero(reach)
    d, _ = cKDTree(xy).query(np.stack([(xs + 0.5) * RES, (ys + 0.5) * RES], 1))
    return float((d <= radius).mean())


@pytest.mark.parametrize("which", ["room", "office"])
def test_serial_float32_program_agrees_with_the_workload_generator(which):
    g = workloads.make_room(1000) if which == "room" else workloads.make_office(1001)[:256, :256]
    clr = workloads.clearance_table(g, RES)
    p0 = workloads.free_start(g, RES, R_ROBOT, 7, clr)
    rho = math.sqrt(float((clr >= R_ROBOT).sum()) * RES * RES / (1.1 * (200 if which == "room" else 600)))
    xy, rounds, nodes = serial_rrt(clr, RES, p0, rho, 0.6, R_ROBOT, 2, 7)
    xs, _, _ = workloads.rrt(g, RES, p0, rho, 0.6, R_ROBOT, 2, 7, clr=clr)
    assert xy.dtype == np.float32 and np.array_equal(xy[0], np.float32(p0))
    assert 0.95 * len(xs) <= len(xy) <= 1.05 * len(xs)
    radius = rho * math.sqrt(2.0)
    assert abs(coverage(xy.astype(np.float64), clr, p0, radius) - coverage(xs, clr, p0, radius)) <= 0.01
    cells = np.floor(xy / np.float32(RES)).astype(np.int64)
    assert (clr[cells[:, 1], cells[:, 0]] >= R_ROBOT).all()
    vox = np.floor(xy / np.float32(rho)).astype(np.int64)
    assert len(np.unique(vox, axis=0)) == len(vox)
    assert rounds >= 2 and nodes >= len(xy)
    again = serial_rrt(clr, RES, p0, rho, 0.6, R_ROBOT, 2, 7)
    assert np.array_equal(again[0], xy) and again[1:] == (rounds, nodes)
