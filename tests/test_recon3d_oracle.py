"""Pins of the oracle's three-dimensional reconstruction with Simpson face
quadrature (grids of one level; `Oracle.stage3d`, `oracle.simpson_flux`).

What fixes it here: the full ghost fill reproduces the periodic global field in
every padded cell (faces, edges, corners); the Simpson flux of a face is the
exact face average of the flux for states quadratic across the face (a shear
whose momentum flux rho u^2 + p the midpoint rule misses by b^2 h^2 / 12), is
the point flux for a uniform face, takes a constant transverse profile at a
local extremum and the monotonized-central line where the parabola would leave
the neighbours' range; one stage keeps a uniform state bit-exact, conserves on
a periodic domain, keeps mirror images bit for bit, reduces to the
dimension-split midpoint scheme when the state varies along one axis only or
when every flux is linear in the state (uniform velocity and temperature), and
refuses grids of several levels; its margin cells (transverse tests near their
thresholds) are the faces a planted near-tie reaches and no others."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import r12 as R

G53 = 5.0 / 3.0
IN = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))
NB = (2, 2, 2)


def _grid(nb=NB, periodic=True):
    return W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / (8 * nb[0]), periodic=(periodic,) * 3)


def test_full_ghost_fill_is_the_periodic_field(oracle_mod):
    G = H.random_smooth_global((16, 16, 16), 3)
    g = _grid()
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts_full(H.scatter(G, NB))
    for s in range(g.n):
        base = np.round(g.origin[s] / g.dx[s]).astype(int) - 3   # global index of padded cell 0 (x, y, z)
        idx = [(base[a] + np.arange(14)) % 16 for a in range(3)]
        expect = G[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
        assert np.array_equal(U[s], expect), s


def test_full_ghost_fill_clamps_at_outflow_boundaries(oracle_mod):
    """On a 3 x 2 x 2 box with outflow boundaries every padded cell (faces,
    edges, corners) holds the global cell at its index clamped to the box,
    axis by axis."""
    nb = (3, 2, 2)
    G = H.random_smooth_global((16, 16, 24), 9)
    g = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / 24, periodic=(False, False, False))
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts_full(H.scatter(G, nb))
    dims = (24, 16, 16)                                       # x, y, z
    for s in range(g.n):
        base = np.round(g.origin[s] / g.dx[s]).astype(int) - 3
        idx = [np.clip(base[a] + np.arange(14), 0, dims[a] - 1) for a in range(3)]
        expect = G[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
        assert np.array_equal(U[s], expect), s


def _face_state(rho, u, p):
    """Conserved state (11) of density rho, x velocity u, pressure p."""
    X = [0.1, 0.2, 0.3, 0.4, 0.5]
    E = p / (G53 - 1.0) + 0.5 * rho * u * u
    tau = (p / (G53 - 1.0)) ** (1.0 / G53)
    return np.array([rho, rho * u, 0.0, 0.0, E, tau] + [rho * x for x in X])


def _averages(rho, u_avg, u2_avg, p):
    """Face-average state of a face cell with rho, p uniform, mean velocity
    u_avg and mean u^2 u2_avg (the energy carries the mean kinetic energy)."""
    A = _face_state(rho, u_avg, p)
    A[4] = p / (G53 - 1.0) + 0.5 * rho * u2_avg
    return A


def test_simpson_flux_is_exact_for_a_transverse_quadratic(oracle_mod):
    """u = U0 + b y across the face (first transverse axis, cells of width 1),
    rho = 1, p = 1, and a first scalar X = X0 + c1 y + c2 y^2 (monotone, with a
    parabola inside its neighbours' range, so unlimited):
      * the x-momentum flux averages rho u^2 + p = U0^2 + b^2 / 12 + 1
        exactly; the point flux of the averaged state misses b^2 / 12;
      * the scalar's flux X u is cubic in y, which the Simpson rule integrates
        exactly when the parabola's point values are exact:
        X0 U0 + (c2 U0 + c1 b) / 12; the midpoint flux misses c1 b / 12."""
    U0, b, p = 0.7, 0.9, 1.0
    X0, c1, c2 = 0.3, 0.1, 0.02
    AL = np.zeros((3, 3, 11))
    for b2 in range(3):
        for b1 in range(3):
            y = float(b1 - 1)
            AL[b2, b1] = _averages(1.0, U0 + b * y, (U0 + b * y) ** 2 + b * b / 12.0, p)
            AL[b2, b1, 6] = X0 + c1 * y + c2 * (y * y + 1.0 / 12.0)
    F, _ = oracle_mod.simpson_flux(AL, AL, 0, eta=0.0)
    exact = U0 ** 2 + b * b / 12.0 + p
    assert F[1] == pytest.approx(exact, rel=1e-14)
    exact_x = X0 * U0 + (c2 * U0 + c1 * b) / 12.0
    assert F[6] == pytest.approx(exact_x, rel=1e-14)
    Fmid, _ = oracle_mod.face_flux(AL[1, 1], AL[1, 1], 0, eta=0.0)
    assert abs(Fmid[1] - exact) > 0.5 * b * b / 12.0
    assert abs(Fmid[6] - exact_x) > 0.5 * c1 * b / 12.0


def test_simpson_flux_of_a_uniform_face_is_the_point_flux(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(3):
        A = _face_state(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(0.5, 2))
        AL = np.broadcast_to(A, (3, 3, 11)).copy()
        B = _face_state(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(0.5, 2))
        AR = np.broadcast_to(B, (3, 3, 11)).copy()
        F, a = oracle_mod.simpson_flux(AL, AR, 0)
        Fp, ap = oracle_mod.face_flux(A, B, 0)
        np.testing.assert_allclose(F, Fp, rtol=4e-16 * 8, atol=1e-300)
        assert a == ap


def test_transverse_limiter(oracle_mod):
    """At a local extremum of the three averages the profile is constant: with
    u = 1, 2, 1 across the face (rho = p = 1, so E = 2, 3.5, 2, also an
    extremum) the momentum flux is that of u = 2, i.e. 4 + 1.  Where the
    parabola would leave the neighbours' range the line with the
    monotonized-central slope min(|a+ - a-| / 2, 2|a0 - a-|, 2|a+ - a0|) takes
    over: u = 0, 0.1, 1 gives the slope 0.2 and points 0, 0.1, 0.2; E = 1.5,
    1.505, 2 gives the slope 0.01 and points 1.5, 1.505, 1.51; the pressures
    (2/3)(E - u^2/2) at the points are 1, 1, 0.99333..., and the Simpson mean
    of u^2 + p is (1 + 4 (0.01 + 1) + (0.04 + 2/3 * 1.49)) / 6."""
    cases = (((1.0, 2.0, 1.0), 5.0),
             ((0.0, 0.1, 1.0), (1.0 + 4.0 * 1.01 + (0.04 + 2.0 / 3.0 * 1.49)) / 6.0))
    for us, expect in cases:
        AL = np.zeros((3, 3, 11))
        for b2 in range(3):
            for b1 in range(3):
                AL[b2, b1] = _face_state(1.0, us[b1], 1.0)
        F, _ = oracle_mod.simpson_flux(AL, AL, 0, eta=0.0)
        assert F[1] == pytest.approx(expect, rel=1e-14), (us, F[1])


def _stage(oracle_mod, G, nb=NB, dt=0.004, threed=True):
    g = _grid(nb)
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts_full(H.scatter(G, nb))
    if threed:
        U1, ms, st = o.stage3d(U, dt)
    else:
        U1, ms, st = o.stage(U, dt)
    assert st == 0
    return U1, U, g


def test_uniform_state_and_conservation(oracle_mod):
    G = H.prim_to_global(*(np.full((16, 16, 16), v) for v in (1.3, 0.2, -0.4, 0.1, 0.8)))
    U1, U, _ = _stage(oracle_mod, G)
    assert np.array_equal(U1[IN], U[IN])
    G = H.random_smooth_global((16, 16, 16), 11)
    U1, U, g = _stage(oracle_mod, G)
    for f in range(W.NF):
        before, absb = H.exact_total(g, U, f)
        after, _ = H.exact_total(g, U1, f)
        assert abs(after - before) <= 1e-13 * absb, f
    assert np.max(np.abs(U1 - U)[IN]) > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(oracle_mod, axis):
    """The transverse parabolas negate their odd part exactly and the Simpson
    sums add the two outer points first, so mirror images agree bit for bit."""
    G = H.random_smooth_global((16, 16, 16), 21 + axis)
    ax = 3 - axis

    def mirror(X):
        M = np.flip(X, axis=ax).copy()
        M[1 + axis] *= -1.0
        return M

    a, _, _ = _stage(oracle_mod, G)
    b, _, _ = _stage(oracle_mod, mirror(G))
    assert np.array_equal(mirror(H.gather(a, NB)), H.gather(b, NB))


def test_one_dimensional_data_is_the_midpoint_scheme(oracle_mod):
    x = (np.arange(16) + 0.5) / 16
    rho = np.broadcast_to(1.0 + 0.3 * np.sin(2 * np.pi * x), (16, 16, 16))
    vx = np.broadcast_to(0.4 * np.cos(2 * np.pi * x), (16, 16, 16))
    p = np.broadcast_to(1.0 + 0.2 * np.sin(4 * np.pi * x), (16, 16, 16))
    z = np.zeros((16, 16, 16))
    G = H.prim_to_global(rho, vx, z, z, p)
    a, _, _ = _stage(oracle_mod, G)
    b, _, _ = _stage(oracle_mod, G, threed=False)
    res = R.r12(a, b)
    assert np.all(res["err"] <= 1e-14), R.summary(res)


def test_flux_linear_states_are_the_midpoint_scheme(oracle_mod):
    """Uniform velocity and an isothermal density wave (p = rho): every
    conserved field but the entropy tracer is proportional to rho, so the
    limiters decide alike, the sound speed and with it the KNP speeds are
    uniform, each flux is linear in the state, and the Simpson rule returns
    the flux of the face averages."""
    x = (np.arange(16) + 0.5) / 16
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = np.broadcast_to(1.0 + 0.3 * np.sin(2 * np.pi * (X + Y)), (16, 16, 16))
    one = np.ones((16, 16, 16))
    G = H.prim_to_global(rho, 0.5 * one, 0.3 * one, 0.0 * one, rho)
    a, _, _ = _stage(oracle_mod, G)
    b, _, _ = _stage(oracle_mod, G, threed=False)
    res = R.r12(a, b)
    assert np.all(res["err"] <= 1e-13), R.summary(res)


def test_grids_of_several_levels_are_refused(oracle_mod):
    w = W.config(3)
    o = oracle_mod.Oracle(w.grid)
    with pytest.raises(ValueError):
        o.fill_ghosts_full(w.state())


def _y_profile_state(ry):
    rho = np.broadcast_to(ry[None, :, None], (16, 16, 16)).copy()
    one = np.ones((16, 16, 16))
    return H.scatter(H.prim_to_global(rho, 0.2 * one, 0.0 * one, 0.0 * one, one), NB)


def _flagged_rows(m):
    rows = set()
    for s in range(8):
        j = (s // 2) % 2
        _, jj, _ = np.nonzero(m[s])
        rows.update((jj + 8 * j).tolist())
    return sorted(rows)


def test_margin_cells_of_the_transverse_tests(oracle_mod):
    """Density varying along y only (uniform u, p): the x- and z-faces see the
    y-profile across them.  A smooth profile puts no transverse test near a
    threshold where it matters.  Rows 4, 5, 6 set to A, A + D, A + 5 D (1 +
    1e-9) give the parabola through those averages an edge value within 1e-9
    D of the row-4 average: a range test within 64 x 2^-24 of its threshold
    (not within 64 x 2^-53), between the parabola and the limited line, whose
    edge values differ by D/2: exactly the x- and z-faces of row 5 are marked
    (16 pencils x 18 face planes x 2 directions = 576) and the cells beside
    them, all in row 5.  With A + 4.5 D in row 6 nothing is near.  (An
    extremum test near its threshold alone is not marked: where one side's
    difference is tiny the parabola leaves the range, and the line's slope is
    at most that difference.)"""
    o = oracle_mod.Oracle(_grid())
    y = np.arange(16)
    ry = 1.0 + 0.3 * np.sin(2 * np.pi * y / 16 + 0.3)
    m, k = o.margin_cells3d(_y_profile_state(ry), 2.0 ** -24)
    assert k == 0 and not m.any()
    A, D = ry[4], 0.05
    ry[5], ry[6] = A + D, A + 5.0 * D * (1.0 + 1e-9)
    m, k = o.margin_cells3d(_y_profile_state(ry), 2.0 ** -24)
    assert k == 576
    assert _flagged_rows(m) == [5]
    assert np.all((m == 0) | (m == R.M_RECON3D))
    m, k = o.margin_cells3d(_y_profile_state(ry), 2.0 ** -53)
    assert k == 0
    ry[6] = A + 4.5 * D
    m, k = o.margin_cells3d(_y_profile_state(ry), 2.0 ** -24)
    assert k == 0
    ry[5], ry[6] = A + 1e-9 * D, A + D      # a near extremum test alone
    m, k = o.margin_cells3d(_y_profile_state(ry), 2.0 ** -24)
    assert 5 not in _flagged_rows(m)
    with pytest.raises(ValueError):
        oracle_mod.Oracle(W.config(3).grid).margin_cells3d(W.config(3).state(), 2.0 ** -24)


@pytest.mark.parametrize("nb,seed", [((1, 1, 1), 3), ((2, 2, 2), 4), ((3, 2, 1), 5)])
def test_numpy_restatement_on_the_global_array(oracle_mod, nb, seed):
    """tests/numpy_stage3d.py states the same stage on the global array of a
    periodic box (neighbours by np.roll: no sub-grids, ghost fill or
    neighbour tables); one blended stage agrees with the oracle bit for bit,
    maximum speed included, on one sub-grid, on 2 x 2 x 2 and on a box with
    unequal sub-grid counts per axis."""
    from tests import numpy_stage3d as N3
    G = H.random_smooth_global((8 * nb[2], 8 * nb[1], 8 * nb[0]), seed)
    g = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / (8 * max(nb)))
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts_full(H.scatter(G, nb))
    _, ms0, _ = o.stage3d(U, 0.0)
    dt = 0.4 / ms0[1]
    G0 = G * (1.0 + 1e-3 * np.sin(np.arange(G.size).reshape(G.shape)))
    U0 = o.fill_ghosts_full(H.scatter(G0, nb))
    ref, ms, st = o.stage3d(U, dt, U0=U0, beta=0.25)
    assert st == 0
    got, amax = N3.stage(G, g.dx[0], dt, G0=G0, beta=0.25)
    assert np.array_equal(H.gather(ref, nb), got)
    assert amax == ms[0]
