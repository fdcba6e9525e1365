"""Seeded synthetic workloads for the batched octree hydro step.

This module builds inputs only: grid descriptors (uniform periodic grids and
2:1-balanced random octrees of 8^3 sub-grids), leaf batches of Zipf-distributed
size, and initial states given as point values at cell centres.  It holds none
of the solver's arithmetic (no reconstruction, flux, update, ghost fill or
reduction); both the CPU oracle and the CUDA library consume what it returns.

Geometry follows the octree description of the paper's Section IV-C: every node
is an N^3 Cartesian sub-grid with N = 8, refined into eight children of twice
the resolution.  Each sub-grid is stored with 3 ghost layers, i.e. a padded
14^3 tile per field, fields in the order

    0 rho, 1 sx, 2 sy, 3 sz, 4 egas (total energy density), 5 tau (entropy
    tracer), 6..10 rho*X_1 .. rho*X_5 (passive scalars),

layout ``U[s][f][k][j][i]`` (x fastest), interior indices 3..10.  Ghost cells
are filled with NaN canaries: each side fills them with its own ghost routine.

Neighbour table ``neighbor[s][face][q]`` (faces -x,+x,-y,+y,-z,+z):
  rel == 0 : q = 0 holds the same-level neighbour (periodic wrap encoded here),
             or -1 for a domain boundary (outflow);
  rel == -1: q = 0 holds the one-level-coarser neighbour; ``octant[s]`` tells
             where this sub-grid sits inside its parent (bit0 x, bit1 y, bit2 z);
  rel == +1: q = t1 + 2*t2 holds the four one-level-finer neighbours touching
             the face, t1/t2 the child offsets along the first/second
             transverse axis (x-face: y,z; y-face: x,z; z-face: x,y).

Random numbers: numpy PCG64, seed 2210064370 + config index (1..5).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

NX = 8          # interior cells per sub-grid edge
NG = 3          # ghost layers
NP = NX + 2 * NG  # padded edge, 14
NF = 11         # conserved fields
GAMMA = 5.0 / 3.0
DE_SWITCH = 1e-3
SEED_BASE = 2210064370

FIELD_NAMES = ("rho", "sx", "sy", "sz", "egas", "tau", "rhoX1", "rhoX2", "rhoX3", "rhoX4", "rhoX5")

# face order: -x, +x, -y, +y, -z, +z ; axis of face = face // 2, side = face % 2
FACE_AXIS = (0, 0, 1, 1, 2, 2)
FACE_SIDE = (0, 1, 0, 1, 0, 1)
TRANSVERSE = ((1, 2), (0, 2), (0, 1))  # transverse axes (first, second) per face axis


@dataclasses.dataclass
class Grid:
    """Grid descriptor: what the oracle and the library both consume."""
    n: int
    dx: np.ndarray            # float64 [n]
    origin: np.ndarray        # float64 [n,3] lower corner of the interior block
    level: np.ndarray         # int8 [n]
    octant: np.ndarray        # int8 [n]
    neighbor: np.ndarray      # int32 [n,6,4]
    neighbor_rel: np.ndarray  # int8 [n,6]
    periodic: bool = False
    gamma: float = GAMMA
    de_switch: float = DE_SWITCH

    def cell_centers(self, ids: Optional[np.ndarray] = None):
        """Cell-centre coordinates of the interior cells, arrays [m,8,8,8] (k,j,i order)."""
        ids = np.arange(self.n) if ids is None else np.asarray(ids)
        o = self.origin[ids]
        h = self.dx[ids]
        c = (np.arange(NX) + 0.5)
        x = o[:, 0, None, None, None] + h[:, None, None, None] * c[None, None, None, :]
        y = o[:, 1, None, None, None] + h[:, None, None, None] * c[None, None, :, None]
        z = o[:, 2, None, None, None] + h[:, None, None, None] * c[None, :, None, None]
        shape = (len(ids), NX, NX, NX)
        return np.broadcast_to(x, shape), np.broadcast_to(y, shape), np.broadcast_to(z, shape)


@dataclasses.dataclass
class Batches:
    """Sub-grid ids in queue order, cut into batches (offsets has n_batches+1 entries)."""
    ids: np.ndarray      # int32 [n_items]
    offsets: np.ndarray  # int32 [n_batches+1]


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    grid: Grid
    batches: Batches
    steps: int
    cfl: float
    precision: str            # "fp64", "mixed" or "both"
    init: Callable[["Workload", Optional[np.ndarray]], np.ndarray]
    description: str = ""

    @property
    def cells(self) -> int:
        return self.grid.n * NX ** 3

    def state(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """Padded initial state, float64 [n,11,14,14,14]; ghosts are NaN canaries."""
        return self.init(self, out)


# ----------------------------------------------------------------------------
# uniform periodic grids
# ----------------------------------------------------------------------------

def uniform_grid(nb: Tuple[int, int, int], lo: Sequence[float], dx: float,
                 periodic: Sequence[bool] = (True, True, True)) -> Grid:
    """Uniform grid of nb[0] x nb[1] x nb[2] sub-grids, x-fastest numbering.

    Non-periodic axes get outflow boundaries (neighbour -1)."""
    bx, by, bz = nb
    n = bx * by * bz
    ids = np.arange(n).reshape(bz, by, bx)
    neighbor = np.full((n, 6, 4), -1, np.int32)
    rel = np.zeros((n, 6), np.int8)
    origin = np.zeros((n, 3))
    for k in range(bz):
        for j in range(by):
            for i in range(bx):
                s = ids[k, j, i]
                origin[s] = (lo[0] + i * NX * dx, lo[1] + j * NX * dx, lo[2] + k * NX * dx)
                pos = [i, j, k]
                dims = [bx, by, bz]
                for face in range(6):
                    a, side = FACE_AXIS[face], FACE_SIDE[face]
                    q = list(pos)
                    q[a] += 1 if side else -1
                    if q[a] < 0 or q[a] >= dims[a]:
                        if not periodic[a]:
                            continue
                        q[a] %= dims[a]
                    neighbor[s, face, 0] = ids[q[2], q[1], q[0]]
    return Grid(n=n, dx=np.full(n, dx), origin=origin, level=np.zeros(n, np.int8),
                octant=np.zeros(n, np.int8), neighbor=neighbor, neighbor_rel=rel,
                periodic=all(periodic))


# ----------------------------------------------------------------------------
# random 2:1-balanced octree
# ----------------------------------------------------------------------------

def _morton(i: int, j: int, k: int, bits: int) -> int:
    code = 0
    for b in range(bits):
        code |= ((i >> b) & 1) << (3 * b) | ((j >> b) & 1) << (3 * b + 1) | ((k >> b) & 1) << (3 * b + 2)
    return code


class _Octree:
    """Leaves keyed by (level, i, j, k); base level 0 has dims nb."""

    def __init__(self, nb, max_level):
        self.nb = tuple(nb)
        self.max_level = max_level
        self.leaves: Dict[Tuple[int, int, int, int], bool] = {}
        for k in range(nb[2]):
            for j in range(nb[1]):
                for i in range(nb[0]):
                    self.leaves[(0, i, j, k)] = True

    def inside(self, lvl, p):
        return all(0 <= p[a] < self.nb[a] << lvl for a in range(3))

    def covering(self, lvl, p):
        """Leaf covering integer position p at level lvl, or None if refined finer."""
        for l in range(lvl, -1, -1):
            sh = lvl - l
            key = (l, p[0] >> sh, p[1] >> sh, p[2] >> sh)
            if key in self.leaves:
                return key
        return None

    def cascade(self, leaf, plan):
        """Append to plan every leaf that must be refined (in order) so that refining
        `leaf` keeps the 2:1 balance across faces, edges and corners."""
        lvl, i, j, k = leaf
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    if di == dj == dk == 0:
                        continue
                    p = (i + di, j + dj, k + dk)
                    if not self.inside(lvl, p):
                        continue
                    c = self.covering(lvl, p)
                    if c is not None and c[0] < lvl and c not in plan:
                        self.cascade(c, plan)
        if leaf not in plan:
            plan.append(leaf)

    def refine(self, leaf):
        del self.leaves[leaf]
        lvl, i, j, k = leaf
        for o in range(8):
            self.leaves[(lvl + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1))] = True


def octree_grid(nb, lo, hi, max_level, n_refine, density: Callable, rng: np.random.Generator,
                draw: int = 64) -> Grid:
    """Seeded random octree with exactly `n_refine` refinements (balance-forced ones
    included), leaves chosen with probability proportional to the mean density over
    the eight octant centres of the leaf.  Leaves are returned in Morton order."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    dx0 = (hi[0] - lo[0]) / (nb[0] * NX)
    assert abs((hi[1] - lo[1]) / (nb[1] * NX) - dx0) < 1e-12 and abs((hi[2] - lo[2]) / (nb[2] * NX) - dx0) < 1e-12
    t = _Octree(nb, max_level)
    done = 0
    off = np.array([[(o & 1), (o >> 1) & 1, (o >> 2) & 1] for o in range(8)], float) * 0.5 + 0.25
    while done < n_refine:
        keys = [key for key in t.leaves if key[0] < max_level]
        arr = np.array(keys, np.int64)
        width = NX * dx0 / (2.0 ** arr[:, 0])
        corner = lo[None, :] + arr[:, 1:4] * width[:, None]
        pts = corner[:, None, :] + off[None, :, :] * width[:, None, None]
        w = density(pts[..., 0], pts[..., 1], pts[..., 2]).mean(axis=1)
        w = w / w.sum()
        picks = rng.choice(len(keys), size=min(draw, len(keys)), replace=True, p=w)
        progressed = False
        for idx in picks:
            if done >= n_refine:
                break
            leaf = tuple(int(v) for v in arr[idx])
            if leaf not in t.leaves:
                continue
            plan: List = []
            t.cascade(leaf, plan)
            if done + len(plan) > n_refine:
                continue
            for p in plan:
                t.refine(p)
            done += len(plan)
            progressed = True
        if not progressed:
            # finish with refinements that need no cascade, in a fixed scan order
            for key in sorted(t.leaves):
                if done >= n_refine:
                    break
                if key[0] >= max_level or key not in t.leaves:
                    continue
                plan = []
                t.cascade(key, plan)
                if len(plan) == 1:
                    t.refine(key)
                    done += 1
    return _grid_from_tree(t, lo, dx0)


def _grid_from_tree(t: _Octree, lo, dx0) -> Grid:
    L = t.max_level
    bits = max(int(math.ceil(math.log2(max(t.nb)))) + L, 1)
    keys = sorted(t.leaves, key=lambda q: (_morton(q[1] << (L - q[0]), q[2] << (L - q[0]), q[3] << (L - q[0]), bits), q[0]))
    index = {key: s for s, key in enumerate(keys)}
    n = len(keys)
    neighbor = np.full((n, 6, 4), -1, np.int32)
    rel = np.zeros((n, 6), np.int8)
    level = np.zeros(n, np.int8)
    octant = np.zeros(n, np.int8)
    origin = np.zeros((n, 3))
    dx = np.zeros(n)
    for s, (lvl, i, j, k) in enumerate(keys):
        level[s] = lvl
        octant[s] = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2) if lvl > 0 else 0
        h = dx0 / (2 ** lvl)
        dx[s] = h
        origin[s] = (lo[0] + i * NX * h, lo[1] + j * NX * h, lo[2] + k * NX * h)
        pos = (i, j, k)
        for face in range(6):
            a, side = FACE_AXIS[face], FACE_SIDE[face]
            p = list(pos)
            p[a] += 1 if side else -1
            if not t.inside(lvl, p):
                continue  # outflow boundary
            key = (lvl, p[0], p[1], p[2])
            if key in t.leaves:
                neighbor[s, face, 0] = index[key]
                continue
            par = (lvl - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1)
            if lvl > 0 and par in t.leaves:
                neighbor[s, face, 0] = index[par]
                rel[s, face] = -1
                continue
            ta, tb = TRANSVERSE[a]
            for t2 in (0, 1):
                for t1 in (0, 1):
                    c = [2 * p[0], 2 * p[1], 2 * p[2]]
                    c[a] += 0 if side else 1   # child half touching our face
                    c[ta] += t1
                    c[tb] += t2
                    ck = (lvl + 1, c[0], c[1], c[2])
                    if ck not in t.leaves:
                        raise RuntimeError("octree is not 2:1 balanced at %r" % (ck,))
                    neighbor[s, face, t1 + 2 * t2] = index[ck]
            rel[s, face] = 1
    return Grid(n=n, dx=dx, origin=origin, level=level, octant=octant, neighbor=neighbor,
                neighbor_rel=rel, periodic=False)


def zipf_batches(n_items: int, s: float, max_size: int, rng: np.random.Generator) -> Batches:
    """Consecutive batches of the queue order with Zipf(s) sizes truncated to [1,max_size]."""
    sizes = []
    left = n_items
    while left > 0:
        z = int(rng.zipf(s))
        while z > max_size:
            z = int(rng.zipf(s))
        z = min(z, left)
        sizes.append(z)
        left -= z
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    return Batches(ids=np.arange(n_items, dtype=np.int32), offsets=offsets)


def single_batch(n: int) -> Batches:
    return Batches(ids=np.arange(n, dtype=np.int32), offsets=np.array([0, n], np.int32))


# ----------------------------------------------------------------------------
# initial states (point values at cell centres)
# ----------------------------------------------------------------------------

def empty_state(n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    if out is None:
        out = np.empty((n, NF, NP, NP, NP))
    out.fill(np.nan)
    return out


def conserved_from_primitive(rho, vx, vy, vz, p, X, gamma=GAMMA):
    """Conserved tuple for an ideal gas: E = p/(gamma-1) + rho|v|^2/2, tau = (p/(gamma-1))^(1/gamma)."""
    eint = p / (gamma - 1.0)
    E = eint + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    tau = eint ** (1.0 / gamma)
    out = [rho, rho * vx, rho * vy, rho * vz, E, tau]
    out += [rho * x for x in X]
    return out


def set_interior(U: np.ndarray, ids, fields) -> None:
    sl = (slice(NG, NG + NX),) * 3
    for f, v in enumerate(fields):
        U[(ids, f) + sl] = v


def _fill_by_chunks(w: Workload, out, fn, chunk=4096):
    U = empty_state(w.grid.n, out)
    for a in range(0, w.grid.n, chunk):
        ids = np.arange(a, min(a + chunk, w.grid.n))
        x, y, z = w.grid.cell_centers(ids)
        set_interior(U, ids, fn(ids, x, y, z))
    return U


def _init_sod(w: Workload, out):
    def fn(ids, x, y, z):
        left = x < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        zero = np.zeros_like(rho)
        X = [left.astype(float), (~left).astype(float), zero, zero, zero]
        return conserved_from_primitive(rho, zero, zero, zero, p, X)
    return _fill_by_chunks(w, out, fn)


def _smooth_periodic(g: np.ndarray, sigma: float) -> np.ndarray:
    k = [np.fft.fftfreq(m) for m in g.shape]
    kz, ky, kx = np.meshgrid(*k, indexing="ij")
    kern = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    return np.real(np.fft.ifftn(np.fft.fftn(g) * kern))


def _init_lognormal(w: Workload, out):
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + w.index))
    bx = int(round(w.grid.n ** (1.0 / 3.0)))    # sub-grids per edge of the periodic cube
    m = bx * NX
    g = rng.standard_normal((m, m, m))          # [z][y][x]
    g = _smooth_periodic(g, 2.0)
    g = (g - g.mean()) / g.std()
    rho_c = np.exp(0.3 * g - 0.045)
    u = rng.uniform(-0.5, 0.5, (3, m, m, m))
    X = rng.uniform(0.0, 1.0, (5, m, m, m))
    U = empty_state(w.grid.n, out)
    for s in range(w.grid.n):
        i, j, k = s % bx, (s // bx) % bx, s // (bx * bx)
        sl = (slice(k * NX, (k + 1) * NX), slice(j * NX, (j + 1) * NX), slice(i * NX, (i + 1) * NX))
        rho = rho_c[sl]
        p = np.ones_like(rho)
        c = np.sqrt(GAMMA * p / rho)
        fields = conserved_from_primitive(rho, u[0][sl] * c, u[1][sl] * c, u[2][sl] * c, p, [x[sl] for x in X])
        set_interior(U, np.array([s]), [f[None] for f in fields])
    return U


RHO_FLOOR = 1e-10


def polytrope_density(x, y, z, cx=0.0, rho_c=1.0):
    r2 = (x - cx) ** 2 + y ** 2 + z ** 2
    return np.maximum(rho_c * np.maximum(1.0 - r2, 0.0) ** 1.5, RHO_FLOOR)


def _scalars(x, y, z, star1, star2):
    X = [star1.astype(float), star2.astype(float)]
    for kk in range(3):
        X.append(0.5 + 0.4 * np.sin(np.pi * (x + 0.3 * kk)) * np.cos(np.pi * (y - 0.2 * kk)))
    return X


def _init_polytrope(perturb: bool):
    def init(w: Workload, out):
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + w.index + 1000))

        def fn(ids, x, y, z):
            rho = polytrope_density(x, y, z)
            p = rho ** GAMMA
            if perturb:
                rho = rho * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, rho.shape))
            R = np.sqrt(x * x + y * y)
            # softened Keplerian profile, tapered smoothly to rest in the
            # low-density envelope (a hard cut at the surface makes face
            # velocities s/rho of the conserved-variable reconstruction blow up)
            vphi = 0.5 * (R / 0.2) / (1.0 + (R / 0.2) ** 2) ** 0.75 * (rho / (rho + 1e-2))
            Rs = np.where(R > 0, R, 1.0)
            vx = np.where(R > 0, -vphi * y / Rs, 0.0)
            vy = np.where(R > 0, vphi * x / Rs, 0.0)
            vz = np.zeros_like(rho)
            star = rho > 1e-9
            return conserved_from_primitive(rho, vx, vy, vz, p, _scalars(x, y, z, star, np.zeros_like(star)))
        return _fill_by_chunks(w, out, fn)
    return init


def binary_density(x, y, z):
    return np.maximum(polytrope_density(x, y, z, -1.5, 1.0), polytrope_density(x, y, z, 1.5, 0.7))


def _init_binary(w: Workload, out):
    def fn(ids, x, y, z):
        rho1 = polytrope_density(x, y, z, -1.5, 1.0)
        rho2 = polytrope_density(x, y, z, 1.5, 0.7)
        rho = np.maximum(rho1, rho2)
        p = rho ** GAMMA
        zero = np.zeros_like(rho)
        return conserved_from_primitive(rho, zero, zero, zero, p, _scalars(x, y, z, rho1 > 1e-9, rho2 > 1e-9))
    return _fill_by_chunks(w, out, fn)


# ----------------------------------------------------------------------------
# the five configurations
# ----------------------------------------------------------------------------

def _rng(index):
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


_CACHE: Dict[int, Workload] = {}


def config(index: int) -> Workload:
    """Configurations 1..5 of the benchmark ladder (grid, batches, recipe); 6 is a
    reduced copy of 5 for profiling; 7 a periodic box of one level for the
    three-dimensional reconstruction."""
    if index in _CACHE:
        return _CACHE[index]
    if index == 1:
        g = uniform_grid((2, 2, 2), (0.0, 0.0, 0.0), 1.0 / 16)
        w = Workload("sod16", 1, g, single_batch(g.n), steps=20, cfl=0.4, precision="fp64", init=_init_sod,
                     description="8 sub-grids, 16^3 periodic, Sod along x")
    elif index == 2:
        g = uniform_grid((8, 8, 8), (0.0, 0.0, 0.0), 1.0 / 64)
        w = Workload("lognormal64", 2, g, single_batch(g.n), steps=10, cfl=0.4, precision="fp64",
                     init=_init_lognormal, description="512 sub-grids, 64^3 periodic, smoothed lognormal density")
    elif index in (3, 4):
        rng = _rng(index)
        nref = 512 if index == 3 else 4608
        g = octree_grid((8, 8, 8), (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0), 3, nref,
                        lambda x, y, z: polytrope_density(x, y, z), rng)
        b = zipf_batches(g.n, 1.1, 512, rng)
        if index == 3:
            w = Workload("polytrope4k", 3, g, b, steps=5, cfl=0.4, precision="fp64", init=_init_polytrope(False),
                         description="4096-leaf octree (levels 0-3), rotating n=1.5 polytrope")
        else:
            w = Workload("polytrope32k", 4, g, b, steps=5, cfl=0.4, precision="mixed", init=_init_polytrope(True),
                         description="32768-leaf octree, polytrope with 1% density perturbation")
    elif index == 5:
        rng = _rng(index)
        g = octree_grid((8, 4, 4), (-4.0, -2.0, -2.0), (4.0, 2.0, 2.0), 4, 9344, binary_density, rng)
        b = zipf_batches(g.n, 1.1, 1024, rng)
        w = Workload("binary64k", 5, g, b, steps=5, cfl=0.4, precision="both", init=_init_binary,
                     description="65536-leaf octree (levels 0-4), two polytropes, mass ratio 0.7")
    elif index == 6:
        # a reduced copy of configuration 5 (same domain, recipe and leaf-batch law,
        # 4096 leaves, levels 0-4) whose state fits in a few GB: the size used for
        # hardware-counter profiles of the kernels
        rng = _rng(index)
        g = octree_grid((8, 4, 4), (-4.0, -2.0, -2.0), (4.0, 2.0, 2.0), 4, 567, binary_density, rng)
        b = zipf_batches(g.n, 1.1, 1024, rng)
        w = Workload("binary4k", 6, g, b, steps=5, cfl=0.4, precision="both", init=_init_binary,
                     description="4097-leaf reduced binary octree (levels 0-4) for profiling")
    elif index == 7:
        # a periodic box of one level at the size of the profiling octree: the
        # measurement case of the three-dimensional reconstruction, which takes
        # grids of one level only
        g = uniform_grid((16, 16, 16), (0.0, 0.0, 0.0), 1.0 / 128)
        w = Workload("lognormal128", 7, g, single_batch(g.n), steps=3, cfl=0.4, precision="fp64",
                     init=_init_lognormal, description="4096 sub-grids, 128^3 periodic, smoothed lognormal density")
    else:
        raise ValueError("configs are numbered 1..7")
    _CACHE[index] = w
    return w
