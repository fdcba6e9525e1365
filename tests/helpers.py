"""Shared test helpers: global<->sub-grid layout moves and a time-step driver.

Only data movement, seeded input recipes and the lagged-CFL driver live here;
no solver arithmetic.
"""
import math

import numpy as np

from paper_2210_06437_gb300 import workloads as W

NX, NG, NP, NF = W.NX, W.NG, W.NP, W.NF


def scatter(G, nb):
    """Global array G[f][Z][Y][X] -> padded sub-grid state (x-fastest sub-grid ids), NaN ghosts."""
    bx, by, bz = nb
    U = W.empty_state(bx * by * bz)
    for k in range(bz):
        for j in range(by):
            for i in range(bx):
                s = (k * by + j) * bx + i
                U[s, :, NG:NG + NX, NG:NG + NX, NG:NG + NX] = G[:, k * NX:(k + 1) * NX, j * NX:(j + 1) * NX,
                                                              i * NX:(i + 1) * NX]
    return U


def gather(U, nb):
    bx, by, bz = nb
    G = np.empty((U.shape[1], bz * NX, by * NX, bx * NX))
    for k in range(bz):
        for j in range(by):
            for i in range(bx):
                s = (k * by + j) * bx + i
                G[:, k * NX:(k + 1) * NX, j * NX:(j + 1) * NX, i * NX:(i + 1) * NX] = U[s, :, NG:NG + NX, NG:NG + NX,
                                                                                      NG:NG + NX]
    return G


def prim_to_global(rho, vx, vy, vz, p, X=None, gamma=W.GAMMA):
    X = X if X is not None else [np.zeros_like(rho)] * 5
    return np.stack(W.conserved_from_primitive(rho, vx, vy, vz, p, X, gamma))


def random_smooth_global(shape, seed, amp=0.2, vamp=0.3):
    """Random smooth periodic primitive state on a global grid of shape (Z, Y, X)."""
    rho, vx, vy, vz, p, Xs = random_smooth_primitives(shape, seed, amp, vamp)
    return prim_to_global(rho, vx, vy, vz, p, Xs)


def random_smooth_primitives(shape, seed, amp=0.2, vamp=0.3):
    """(rho, vx, vy, vz, p, [X1..X5]) of random_smooth_global."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z, Y, X = shape
    z, y, x = np.meshgrid(np.arange(Z) / Z, np.arange(Y) / Y, np.arange(X) / X, indexing="ij")

    def smooth():
        a = rng.uniform(-1, 1, 6)
        return (np.sin(2 * np.pi * (x + a[0])) * np.cos(2 * np.pi * (y + a[1])) +
                np.sin(2 * np.pi * (z + a[2])) * np.cos(2 * np.pi * (x + a[3])) +
                0.5 * np.sin(4 * np.pi * (y + a[4]) + 2 * np.pi * z * a[5]))
    rho = 1.0 + amp * smooth()
    p = 1.0 + amp * smooth()
    v = [vamp * smooth() for _ in range(3)]
    Xs = [0.5 + 0.3 * smooth() / 2.5 for _ in range(5)]
    return rho, v[0], v[1], v[2], p, Xs


def advance(o, U, t_end, cfl, max_steps=100000):
    """Lagged-CFL SSP-RK3 driver on the oracle: the first dt from a dry stage on the
    initial state, later ones from stage 1 of the previous step; the last step is cut
    to land on t_end.  Returns (U, t, steps)."""
    o.fill_ghosts(U)
    _, ms, st = o.stage(U, 0.0)
    assert st == 0
    t, n = 0.0, 0
    while t < t_end - 1e-15 and n < max_steps:
        dt = min(cfl / ms[1], t_end - t)
        U, ms, st = o.rk3_step(U, dt)
        assert st == 0
        t += dt
        n += 1
    return U, t, n


def exact_total(grid, U, f):
    """Correctly rounded sum of dx^3 * U_f over all interior cells (math.fsum)."""
    terms = (U[:, f, NG:NG + NX, NG:NG + NX, NG:NG + NX] * (grid.dx ** 3)[:, None, None, None]).ravel()
    return math.fsum(terms.tolist()), math.fsum(np.abs(terms).tolist())


def quasi_1d_grid(nx_sub, dx, periodic_x):
    return W.uniform_grid((nx_sub, 1, 1), (0.0, 0.0, 0.0), dx, periodic=(periodic_x, True, True))


def amr_blob_state(seed=3):
    """Small outflow octree refined around a blob; density, velocity and
    scalars vary inside |r| < 0.6 and are uniform (velocity zero) outside, so
    nothing crosses the domain boundary."""
    R = 0.6

    def bump(x, y, z):
        r2 = (x * x + y * y + z * z) / (R * R)
        return np.where(r2 < 1.0, (1.0 - r2) ** 3, 0.0)

    rng = np.random.Generator(np.random.PCG64(seed))
    g = W.octree_grid((2, 2, 2), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), 2, 9,
                      lambda x, y, z: 0.05 + bump(x, y, z), rng)
    U = W.empty_state(g.n)
    c = (np.arange(W.NX) + 0.5)
    for s in range(g.n):
        o, h = g.origin[s], g.dx[s]
        z, y, x = np.meshgrid(o[2] + c * h, o[1] + c * h, o[0] + c * h, indexing="ij")
        b = bump(x, y, z)
        rho = 1.0 + 0.5 * b
        vx, vy, vz = (-0.6 * y + 0.3) * b, (0.6 * x - 0.2) * b, 0.4 * b
        X = [b, 1.0 - b, 0.5 * b, np.zeros_like(b), np.zeros_like(b)]
        U[s, :, W.NG:W.NG + W.NX, W.NG:W.NG + W.NX, W.NG:W.NG + W.NX] = np.stack(
            W.conserved_from_primitive(rho, vx, vy, vz, np.ones_like(b), X))
    return g, U


def neighbours(grid, ids):
    """Global ids read across the faces of sub-grids ids (same level, coarser, finer)."""
    nb = grid.neighbor[ids]
    rel = grid.neighbor_rel[ids]
    used = np.zeros_like(nb, dtype=bool)
    used[:, :, 0] = nb[:, :, 0] >= 0
    used[:, :, 1:] = (rel == 1)[:, :, None]
    return np.unique(nb[used])


def cone_grid(grid, sample, rings):
    """A standalone grid made of `sample` and `rings` rings of face neighbours
    around it (faces leaving the set become outflow).  Returns (local grid,
    global ids in local order, local index of every ring: list of arrays, ring
    0 = sample).  An RK stage computed on the local grid is exact on ring r
    when its input is exact on ring r + 1."""
    rings_g = [np.unique(np.asarray(sample, np.int64))]
    for _ in range(rings):
        rings_g.append(np.union1d(rings_g[-1], neighbours(grid, rings_g[-1])))
    gids = rings_g[-1]
    lut = np.full(grid.n, -1, np.int64)
    lut[gids] = np.arange(len(gids))
    nb = grid.neighbor[gids]
    rel = grid.neighbor_rel[gids].copy()
    loc = np.where(nb >= 0, lut[np.maximum(nb, 0)], -1).astype(np.int32)
    # a face whose neighbours are not all local becomes outflow
    for r in range(len(gids)):
        for f in range(6):
            k = 4 if rel[r, f] == 1 else 1
            if np.any(loc[r, f, :k] < 0):
                loc[r, f, :] = -1
                rel[r, f] = 0
            elif rel[r, f] != 1:
                loc[r, f, 1:] = -1
    g = W.Grid(n=len(gids), dx=grid.dx[gids].copy(), origin=grid.origin[gids].copy(), level=grid.level[gids].copy(),
               octant=grid.octant[gids].copy(), neighbor=loc, neighbor_rel=rel, periodic=False, gamma=grid.gamma,
               de_switch=grid.de_switch)
    return g, gids, [lut[r] for r in rings_g]


def resync_case(seed=11):
    """Periodic 2x2x2 sub-grids (16^3 cells): a random smooth state whose tracer
    is scrambled (no longer matching the internal energy), with a slab of cold
    fast cells (x < 4: speed 3, pressure 1e-6, internal energy about 1e-6 of
    the total, below the dual-energy switch).  Returns (grid, U, cold mask
    [8, 14, 14, 14] of the padded cells)."""
    rho, vx, vy, vz, p, Xs = random_smooth_primitives((16, 16, 16), seed)
    cold = np.zeros(rho.shape, bool)
    cold[:, :, :4] = True
    vx = np.where(cold, 3.0, vx)
    p = np.where(cold, 1e-6, p)
    G = prim_to_global(rho, vx, vy, vz, p, Xs)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    G[5] *= rng.uniform(0.5, 1.5, G[5].shape)
    grid = W.uniform_grid((2, 2, 2), (0.0, 0.0, 0.0), 1.0 / 16, periodic=(True, True, True))
    return grid, scatter(G, (2, 2, 2)), scatter(cold[None].astype(float), (2, 2, 2))[:, 0] > 0.5
