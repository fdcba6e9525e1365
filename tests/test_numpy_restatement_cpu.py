"""The oracle against a second, independent NumPy statement of one stage
(tests/numpy_stage.py), on 1-8 same-level sub-grids with random smooth states,
periodic and outflow boundaries, and one blended stage; and the 1-D reduction:
y,z-uniform data give the same rows as the NumPy scheme on a single line.
Both follow the definition's order of operations, so they agree to the last
bit or within a few ulps of the per-cell values (R12 <= 1e-14)."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import numpy_stage as NS
from tests import r12 as R


def _case(nb, periodic, seed):
    shape = (nb[2] * 8, nb[1] * 8, nb[0] * 8)
    G = H.random_smooth_global(shape, seed)
    grid = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / 16, periodic=(periodic,) * 3)
    return grid, H.scatter(G, nb)


@pytest.mark.parametrize("nb,periodic", [((1, 1, 1), True), ((2, 1, 1), False), ((2, 2, 2), True),
                                         ((2, 2, 1), False)])
def test_oracle_stage_equals_numpy_restatement(oracle_mod, nb, periodic):
    grid, U = _case(nb, periodic, 70 + sum(nb))
    o = oracle_mod.Oracle(grid)
    o.fill_ghosts(U)
    _, ms, st = o.stage(U, 0.0)
    dt = 0.4 / ms[1]
    ref, ms_o, st = o.stage(U, dt)
    assert st == 0
    got, amax = NS.stage(U, grid.dx, dt, grid.gamma, grid.de_switch)
    res = R.r12(got, ref)
    assert np.all(res["err"] <= 1e-14), R.summary(res)
    assert abs(amax.max() - ms_o[0]) <= 1e-15 * ms_o[0]
    # a blended stage (beta = 2/3 against a perturbed U0)
    U0 = U.copy()
    U0[R.SL] *= 1.0 + 1e-3 * np.sin(np.arange(U0[R.SL].size).reshape(U0[R.SL].shape))
    ref2, _, _ = o.stage(U, dt, U0=U0, beta=2.0 / 3.0)
    got2, _ = NS.stage(U, grid.dx, dt, grid.gamma, grid.de_switch, U0=U0, beta=2.0 / 3.0)
    res2 = R.r12(got2, ref2)
    assert np.all(res2["err"] <= 1e-14), R.summary(res2)


def test_one_dimensional_reduction_matches_a_single_line(oracle_mod):
    """y,z-uniform data on 4 x 1 x 1 outflow sub-grids: every row of the
    oracle's result equals the NumPy scheme applied to one line of 32 cells
    padded by outflow copies (transverse fluxes cancel exactly)."""
    nx = 32
    x = (np.arange(nx) + 0.5) / nx
    rho = 1.0 + 0.3 * np.exp(-((x - 0.4) / 0.1) ** 2)
    vx = 0.4 * np.sin(2 * np.pi * x)
    p = 1.0 + 0.2 * np.cos(2 * np.pi * x)
    sh = (8, 8, nx)
    b = lambda a: np.broadcast_to(a, sh).copy()
    G = H.prim_to_global(b(rho), b(vx), np.zeros(sh), np.zeros(sh), b(p), [b(0.5 + 0.2 * x)] * 5)
    nb = (4, 1, 1)
    grid = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / nx, periodic=(False, True, True))
    U = H.scatter(G, nb)
    o = oracle_mod.Oracle(grid)
    o.fill_ghosts(U)
    _, ms, _ = o.stage(U, 0.0)
    dt = 0.4 / ms[1]
    ref, _, _ = o.stage(U, dt)
    Gr = H.gather(ref, nb)
    assert np.all(Gr == Gr[:, :1, :1, :])            # identical rows
    # the line: 32 cells + 3 outflow ghosts on each side, as one pencil of a
    # 1 x 1 x 1 "sub-grid" in x whose transverse neighbours are itself
    line = np.concatenate([np.repeat(G[:, 0, 0, :1], 3, axis=1), G[:, 0, 0, :], np.repeat(G[:, 0, 0, -1:], 3, axis=1)],
                          axis=1)                      # [11, 38]
    got = np.empty((11, nx))
    for c0 in range(0, nx, 8):                       # sub-grids of 8 cells, pencils of 14
        q = line[:, c0:c0 + 14]
        aL, aR = NS.ppm(q)
        F, _ = NS.flux(aR[:, 2:11], aL[:, 3:12], 0, grid.gamma, grid.de_switch)
        got[:, c0:c0 + 8] = q[:, 3:11] + (dt / grid.dx[0]) * (F[:, 0:8] - F[:, 1:9])
    row = Gr[:, 0, 0, :]
    den = np.maximum(np.abs(row), 1e-8 * np.abs(row).max(axis=1, keepdims=True))
    diff = np.abs(got - row)
    d = np.where(den > 0, diff / np.where(den > 0, den, 1.0), np.where(diff == 0, 0.0, np.inf))
    assert d.max() <= 1e-14, d.max()
