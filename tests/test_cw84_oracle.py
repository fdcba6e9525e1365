"""Pins of the oracle's CW84 PPM extensions (Oracle(cw84=...)): shock flattening
(Colella & Woodward 1984, Section 4) and contact steepening (eqs. 1.14-1.17),
both coefficients properties of the cell applied to every conserved field.
What fixes them here: the fourth ghost layer that flattening reads follows the
ghost-fill geometry (same level, coarse injection, fine mean, outflow) on a
linear field; where the detectors stay off (smooth, well-resolved data) the
scheme is the base PPM bit for bit; on the Sod tube the extensions lower the
L1 error of the density against the exact Riemann solution and flattening
removes post-shock oscillation (total variation closer to the exact 0.875),
with no new extrema; a contact advected for one period stays sharper with
steepening (within 10 % of its initial bounds) and with an unchanged signal speed; the
extended scheme keeps uniform states, mirror images and conservation exact."""
import math

import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import riemann_exact as R

G53 = 5.0 / 3.0
IN = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))
ALL = 3


def _linear(x, y, z):
    return 0.7 + 1.3 * x - 0.4 * y + 2.1 * z


def test_fourth_ghost_layer_geometry(oracle_mod):
    """The fourth layer (the one flattening adds) by the same rules as the three
    filled ones: a linear field is reproduced at the ghost centre (same level),
    at the centre of the coarse cell containing it (coarser neighbour), as the
    mean of the 8 fine centres (finer: the coarse centre), or as the nearest
    interior cell (outflow)."""
    w = W.config(3)
    g = w.grid
    U = W.empty_state(g.n)
    x, y, z = g.cell_centers()
    U[:, 2, 3:11, 3:11, 3:11] = _linear(x, y, z)
    o = oracle_mod.Oracle(g)
    rng = np.random.default_rng(4)
    seen = {-1: 0, 0: 0, 1: 0, "out": 0}
    for s in rng.choice(g.n, 300, replace=False):
        for face in range(6):
            a, side = W.FACE_AXIS[face], W.FACE_SIDE[face]
            b1, b2 = W.TRANSVERSE[a]
            rel, nb0 = g.neighbor_rel[s, face], g.neighbor[s, face, 0]
            ga = W.NX + 3 if side else -4
            for c1 in (0, 3, 6):
                for c2 in (1, 5, 7):
                    idx = [0, 0, 0]
                    idx[a], idx[b1], idx[b2] = ga, c1, c2
                    pc = g.origin[s] + (np.array(idx) + 0.5) * g.dx[s]
                    val = o.ghost_cell(U, s, face, ga, c1, c2, 2)
                    if nb0 < 0:
                        jdx = list(idx)
                        jdx[a] = 7 if side else 0
                        expect = U[s, 2, jdx[2] + 3, jdx[1] + 3, jdx[0] + 3]
                        seen["out"] += 1
                    elif rel == -1:
                        h = g.dx[nb0]
                        ci = np.floor((pc - g.origin[nb0]) / h)
                        assert np.all(ci >= 0) and np.all(ci < 8)
                        expect = _linear(*(g.origin[nb0] + (ci + 0.5) * h))
                        seen[-1] += 1
                    else:
                        expect = _linear(*pc)
                        seen[int(rel)] += 1
                    assert val == pytest.approx(expect, rel=1e-14, abs=1e-13), (s, face, rel, c1, c2)
    assert all(v > 0 for v in seen.values()), seen


def _run_1d(oracle_mod, ncell, cw84, rho, vx, p, t_end, periodic):
    nsub = ncell // 8
    dx = 1.0 / ncell
    g = H.quasi_1d_grid(nsub, dx, periodic_x=periodic)
    sh = (8, 8, ncell)
    z = np.zeros(sh)
    G = H.prim_to_global(np.broadcast_to(rho, sh), np.broadcast_to(vx, sh), z, z, np.broadcast_to(p, sh))
    o = oracle_mod.Oracle(g, cw84=cw84)
    U, t, n = H.advance(o, H.scatter(G, (nsub, 1, 1)), t_end, 0.4)
    out = H.gather(U, (nsub, 1, 1))
    return out[0, 4, 4, :], n


def _sod(oracle_mod, ncell, cw84):
    x = (np.arange(ncell) + 0.5) / ncell
    left = x < 0.5
    r, _ = _run_1d(oracle_mod, ncell, cw84, np.where(left, 1.0, 0.125), 0.0, np.where(left, 1.0, 0.1), 0.2, False)
    rex, _, _ = R.sample((x - 0.5) / 0.2, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, G53)
    return np.sum(np.abs(r - rex)) / ncell, np.sum(np.abs(np.diff(r))), r


@pytest.mark.parametrize("ncell", [128, 256])
def test_sod_tube_with_extensions(oracle_mod, ncell):
    # measured once: L1(rho) base 5.52e-3 / 2.75e-3; flattening and steepening
    # 5.00e-3 / 2.47e-3; total variation (exact 0.875) base 0.8936 / 0.8926,
    # flattening alone 0.8865 / 0.8858
    e0, tv0, r0 = _sod(oracle_mod, ncell, 0)
    e3, tv3, r3 = _sod(oracle_mod, ncell, ALL)
    _, tv1, r1 = _sod(oracle_mod, ncell, 1)
    assert e3 < 0.93 * e0, (e0, e3)
    assert tv1 < tv0 - 0.005, (tv0, tv1)
    for r in (r1, r3):   # no new extrema
        assert r.max() <= 1.0 + 1e-12 and r.min() >= 0.125 - 1e-12


def test_contact_stays_sharper_with_steepening(oracle_mod):
    ncell = 128
    x = (np.arange(ncell) + 0.5) / ncell
    inside = (x > 0.25) & (x < 0.75)
    rho = np.where(inside, 1.0, 0.1)
    out = {}
    for cw in (0, 2):
        r, n = _run_1d(oracle_mod, ncell, cw, rho, 1.0, 1.0, 1.0, True)
        width = int(np.sum((r > 0.145) & (r < 0.955)))   # cells inside the 5..95 % band
        out[cw] = (np.sum(np.abs(r - rho)) / ncell, width, n, r)
    (e0, w0, n0, _), (e2, w2, n2, r2) = out[0], out[2]
    # measured once: width 13 -> 10 cells, L1 2.09e-2 -> 1.89e-2, steps 1641 -> 1708;
    # after the full period the steepened profile over- and undershoots (max
    # 1.0375, min 0.0922: wiggles of a few per cent spread through the low
    # plateau) where the base scheme stays inside [0.1, 1]: the cost of
    # steepening every conserved field
    assert w2 < w0 and e2 < e0, (w0, w2, e0, e2)
    assert r2.max() <= 1.05 and r2.min() >= 0.09
    assert abs(n2 - n0) <= 0.1 * n0   # no spurious signal speed at the contact


def _wave(ncell):
    xl = np.arange(ncell) / ncell
    dx = 1.0 / ncell
    return 1.0 + 0.2 * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * (xl + dx))) / (2 * np.pi * dx)


def test_smooth_wave_is_the_base_scheme_bit_for_bit(oracle_mod):
    """No shock (uniform pressure, no compression) and a resolved wave
    (steepening's eta-tilde ~ (k dx)^2 / 6 below eta2): the detectors stay off."""
    rho = _wave(64)
    a, _ = _run_1d(oracle_mod, 64, 0, rho, 1.0, 1.0, 0.25, True)
    b, _ = _run_1d(oracle_mod, 64, ALL, rho, 1.0, 1.0, 0.25, True)
    assert np.array_equal(a, b)


def _step3d(oracle_mod, G, cw84, nb=(2, 2, 2), dt=0.004):
    g = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / 16)
    o = oracle_mod.Oracle(g, cw84=cw84)
    U = o.fill_ghosts(H.scatter(G, nb))
    U1, ms, st = o.rk3_step(U, dt)
    assert st == 0
    return H.gather(U1, nb), g, U, U1


def _blast(seed):
    """A pressure jump with converging flow (both detectors fire) plus noise."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(16) + 0.5,) * 3, indexing="ij")
    r2 = (x - 8) ** 2 + (y - 7.5) ** 2 + (z - 8.5) ** 2
    p = np.where(r2 < 16, 10.0, 1.0) * (1 + 0.01 * rng.standard_normal((16, 16, 16)))
    rho = np.where(r2 < 9, 2.0, 1.0) * (1 + 0.01 * rng.standard_normal((16, 16, 16)))
    v = [-0.3 * (c - 8) / 8 for c in (x, y, z)]
    return H.prim_to_global(rho, *v, p)


def test_extensions_fire_and_keep_the_invariants(oracle_mod):
    G = _blast(5)
    base, _, _, _ = _step3d(oracle_mod, G, 0)
    ext, g, U, U1 = _step3d(oracle_mod, G, ALL)
    assert not np.array_equal(base, ext)          # the detectors fired
    for f in range(W.NF):                          # periodic: conservation
        before, absb = H.exact_total(g, U, f)
        after, _ = H.exact_total(g, U1, f)
        assert abs(after - before) <= 1e-13 * absb, (f, after - before)
    for axis in range(3):                          # mirror images, bit for bit
        ax = 3 - axis
        M = np.flip(G, axis=ax).copy()
        M[1 + axis] *= -1.0
        outm, _, _, _ = _step3d(oracle_mod, M, ALL)
        back = np.flip(outm, axis=ax).copy()
        back[1 + axis] *= -1.0
        assert np.array_equal(back, ext), axis
    rng = np.random.default_rng(9)                 # uniform states
    for _ in range(2):
        u = [rng.uniform(0.2, 2)] + list(rng.uniform(-1, 1, 3)) + [rng.uniform(0.2, 2)]
        Gu = H.prim_to_global(*(np.full((16, 16, 16), c) for c in u))
        out, _, _, _ = _step3d(oracle_mod, Gu, ALL)
        assert np.array_equal(out, Gu)
