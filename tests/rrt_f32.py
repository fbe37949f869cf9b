"""Algorithm 1 (Sec. III-A), one point at a time, in float32: test
infrastructure for the GPU sampler, which must grow exactly this tree.

The steps are Algorithm 1's: per round, N_sampling = ceil(W H res^2 / rho^2)
random points; each extends from its nearest node (squared distance, ties to
the lower index) by min(eta, distance), eta from the clearance at that node
(AdaptiveExpandDist: eta_max at >= 2 r_robot, r_robot at <= r_robot, linear
between); the new point must lie in the map and every point of the segment at
spacing res / 2, both ends included, must have clearance >= r_robot; a voxel
of side rho keeps its first node; a round that adds at most eps_gain voxels
ends the sampling.  The random points come from the counter-based splitmix64
generator (Steele, Lea and Flood, 2014) keyed by (seed, round, index, axis),
which both sides implement from its published definition.  Every arithmetic
step is a single float32 operation, rounded once, as numpy does it.
"""
import math

import numpy as np

F = np.float32
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def unit_draw(seed: int, rnd: int, i: int, k: int) -> np.float32:
    """A uniform draw in [0, 1): the top 53 bits of the hash, rounded to float32."""
    c = (seed ^ ((rnd << 40) | (i << 1) | k)) & _M64
    return F((splitmix64(c) >> 11) * (1.0 / 9007199254740992.0))


def serial_rrt(clr, res, p0, rho, eta_max=0.6, r_robot=0.21, eps_gain=2, seed=0, max_rounds=500,
               node_cap=4_000_000):
    """Returns (representatives float32 [n, 2] in node order, rounds, nodes)."""
    H, W = clr.shape
    fres, frho, feta, frr = F(res), F(rho), F(eta_max), F(r_robot)
    Wm, Hm = F(W) * fres, F(H) * fres
    n_s = math.ceil(W * H * res * res / (rho * rho))
    vw = math.ceil(W * res / rho) + 1
    half = F(0.5) * fres

    def clearance(x, y):   # x, y float32 arrays
        cx = np.floor(x / fres).astype(np.int64)
        cy = np.floor(y / fres).astype(np.int64)
        inside = (cx >= 0) & (cy >= 0) & (cx < W) & (cy < H)
        out = np.zeros(np.shape(x), F)
        out[inside] = clr[cy[inside], cx[inside]]
        return out

    def voxel(x, y):
        return int(np.floor(y / frho)) * vw + int(np.floor(x / frho))

    X = np.zeros(min(node_cap, 1 << 16), F)
    Y = np.zeros_like(X)
    C = np.zeros_like(X)
    X[0], Y[0] = F(p0[0]), F(p0[1])
    C[0] = clearance(X[:1], Y[:1])[0]
    n = 1
    claimed = {voxel(X[0], Y[0])}
    reps = [0]
    rounds = 0
    while True:
        gain = 0
        for i in range(n_s):
            rx = unit_draw(seed, rounds, i, 0) * Wm
            ry = unit_draw(seed, rounds, i, 1) * Hm
            ex, ey = X[:n] - rx, Y[:n] - ry
            b = int(np.argmin(ex * ex + ey * ey))
            px, py, dn = X[b], Y[b], C[b]
            if dn >= F(2.0) * frr:
                eta = feta
            elif dn <= frr:
                eta = frr
            else:
                eta = frr + ((feta - frr) * (dn - frr)) / frr
            vx, vy = rx - px, ry - py
            L = np.sqrt(vx * vx + vy * vy)
            if not L > F(0.0):
                continue
            step = min(eta, L)
            nx, ny = px + (vx / L) * step, py + (vy / L) * step
            if not (nx >= F(0.0) and ny >= F(0.0) and nx < Wm and ny < Hm):
                continue
            nseg = int(np.ceil(step / half))
            f = np.arange(nseg + 1, dtype=F) / F(nseg) if nseg else np.zeros(1, F)
            if (clearance(px + (nx - px) * f, py + (ny - py) * f) < frr).any():
                continue
            if n >= node_cap:
                continue
            if n == len(X):
                X, Y, C = (np.concatenate([v, np.zeros_like(v)]) for v in (X, Y, C))
            X[n], Y[n] = nx, ny
            C[n] = clearance(np.array([nx], F), np.array([ny], F))[0]
            v = voxel(nx, ny)
            if v not in claimed:
                claimed.add(v)
                reps.append(n)
                gain += 1
            n += 1
        rounds += 1
        if gain <= eps_gain or rounds >= max_rounds or n >= node_cap:
            break
    idx = np.array(reps)
    return np.stack([X[idx], Y[idx]], 1), rounds, n
