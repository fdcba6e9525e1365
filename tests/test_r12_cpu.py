"""The per-cell error metric (R12) and the oracle's margin cells, on the CPU.

The metric is checked on hand-made arrays whose errors are known; the margin
cells on states where the position of every near-threshold decision is known:
a uniform state has none, a planted pair of nearly equal cells is found at
exactly the cells within 3 of it along its pencil, and a planted dual-energy
face marks the cells around both of its sides.
"""
import numpy as np

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import r12 as R

NG, NX = 3, 8


def test_metric_per_cell_with_floor():
    r = np.ones((1, 11, 8, 8, 8))
    r[0, 0, 0, 0, 0] = 1e-12          # a tiny cell: measured against the floor 1e-8 * max
    x = r.copy()
    x[0, 0, 0, 0, 0] += 1e-14         # 1e-14 / 1e-8 = 1e-6
    x[0, 1, 1, 2, 3] *= 1 + 3e-7      # relative 3e-7
    x[0, 7] = 0.0
    r[0, 7] = 0.0                     # identically zero field, exactly zero: no error
    res = R.r12(x, r)
    assert abs(res["err"][0] - 1e-6) < 1e-12
    assert abs(res["err"][1] - 3e-7) < 1e-12
    assert res["err"][7] == 0.0 and res["err"][2] == 0.0
    assert res["worst"] == (0, 0, 0, 0, 0)
    x[0, 7, 0, 0, 0] = 1e-300         # a zero reference field must stay exactly zero
    assert np.isinf(R.r12(x, r)["err"][7])


def test_metric_dual_energy_margin_cells_are_left_out():
    r = np.ones((2, 11, 8, 8, 8))
    x = r.copy()
    x[1, 4, 5, 5, 5] = 2.0            # a large error in a margin cell
    m = np.zeros((2, 8, 8, 8), np.uint8)
    m[1, 5, 5, 5] = R.M_DUAL
    m[0, 1, 1, 1] = R.M_SLOPE         # near a PPM test only: still gated
    res = R.r12(x, r, m)
    assert res["err"][4] == 0.0 and res["err_margin"][4] == 1.0 and res["err_all"][4] == 1.0
    assert res["n_margin"] == 1 and res["n_near_ppm"] == 1


def _gather_mask(mask, bits):
    """[8 sub-grids, 8, 8, 8] margin mask (x-fastest sub-grid ids) -> global bool [16, 16, 16] of `bits`."""
    g = np.zeros((16, 16, 16), bool)
    for s in range(8):
        i, j, k = s & 1, (s >> 1) & 1, s >> 2
        g[k * 8:(k + 1) * 8, j * 8:(j + 1) * 8, i * 8:(i + 1) * 8] = (mask[s] & bits) != 0
    return g


def _grid_state(G):
    grid = W.uniform_grid((2, 2, 2), (0.0, 0.0, 0.0), 1.0 / 16, periodic=(True, True, True))
    return grid, H.scatter(G, (2, 2, 2))


def test_no_margins_on_a_uniform_state(oracle_mod):
    sh = (16, 16, 16)
    G = H.prim_to_global(*(np.full(sh, v) for v in (1.3, 0.2, -0.1, 0.4, 0.9)))
    grid, U = _grid_state(G)
    o = oracle_mod.Oracle(grid)
    o.fill_ghosts(U)
    for eps in R.EPS.values():
        mask, k = o.margin_cells(U, eps)
        assert k == 0 and not mask.any()


def test_planted_near_slope_is_found_along_its_pencil(oracle_mod):
    # density linear in x; one cell raised so that its right difference is
    # within rounding of zero: the slope tests of cells 4 and 5 are near
    x = np.arange(16.0)
    rho = np.broadcast_to(1.0 + 0.01 * x, (16, 16, 16)).copy()
    rho[:, :, 5] = rho[:, :, 6] * (1 - 1e-9)
    G = H.prim_to_global(rho, *(np.zeros((16, 16, 16)),) * 3, np.ones((16, 16, 16)))
    grid, U = _grid_state(G)
    o = oracle_mod.Oracle(grid)
    o.fill_ghosts(U)
    mask, k = o.margin_cells(U, 2.0 ** -24)
    assert k > 0
    g = _gather_mask(mask, 0xff)   # [z, y, x]
    # only x-pencils see the near test; every row has the same columns marked
    cols = np.flatnonzero(g[0, 0])
    assert np.array_equal(g, np.broadcast_to(np.isin(np.arange(16), cols), g.shape))
    # near tests at global x = 5, 6 (slopes of cells 5, 6 and the parabola of
    # cell 5): the marked cells lie within 3 of them
    assert cols.min() >= 2 and cols.max() <= 9 and {5, 6} <= set(cols)
    slope = _gather_mask(mask, R.M_SLOPE)
    assert slope[0, 0, 2:10].all() and not slope[0, 0, :2].any() and not slope[0, 0, 10:].any()
    # a difference of 1e-9 is far from rounding in FP64: no margin there
    _, k64 = o.margin_cells(U, 2.0 ** -53)
    assert k64 == 0


def test_planted_dual_energy_face_is_found(oracle_mod):
    # uniform density and velocity, internal energy linear in x and equal to
    # eta E exactly at the face x = 8 (between cells 7 and 8): PPM reproduces
    # linear data, so only the two sides of that face sit at the switch, and
    # the cells within 3 of them (x = 4..11) are marked; every other face is
    # 10 % of a cell's change away from the threshold
    sh = (16, 16, 16)
    eta, gamma, ek = 1e-3, 5.0 / 3.0, 4.5
    e8 = ek * eta / (1.0 - eta)
    xc = np.arange(16) + 0.5
    ei = np.broadcast_to(e8 * (1.0 + 0.1 * (xc - 8.0)), sh)
    G = H.prim_to_global(np.ones(sh), np.full(sh, 3.0), np.zeros(sh), np.zeros(sh), (gamma - 1.0) * ei)
    grid, U = _grid_state(G)
    o = oracle_mod.Oracle(grid)
    o.fill_ghosts(U)
    for eps in R.EPS.values():
        mask, k = o.margin_cells(U, eps)
        dual = _gather_mask(mask, R.M_DUAL)
        assert k > 0 and dual[:, :, 4:12].all(), eps
        assert not dual[:, :, :4].any() and not dual[:, :, 12:].any(), eps
