"""Pins of the CPU oracle against what mathematics and textbooks fix (no GPU).

Each test checks the oracle against something other than itself: exactness of
PPM on polynomial data, closed-form fluxes, special cases where the two flux
forms coincide, symmetry and conservation invariants of the scheme, the exact
Riemann solution of the Sod tube, a measured convergence order, and geometry of
the AMR ghost fill.
"""
import functools
import math

import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import riemann_exact as R

G53 = 5.0 / 3.0


# ---------------------------------------------------------------------------
# PPM reconstruction (Colella & Woodward 1984)
# ---------------------------------------------------------------------------

def test_ppm_reproduces_linear_data(oracle_mod):
    m = np.arange(14.0)
    q = 0.3 + 1.7 * m
    aL, aR = oracle_mod.ppm_pencil(q)
    for c in range(2, 12):
        assert aL[c] == pytest.approx(0.3 + 1.7 * (c - 0.5), rel=1e-15, abs=1e-14)
        assert aR[c] == pytest.approx(0.3 + 1.7 * (c + 0.5), rel=1e-15, abs=1e-14)


def test_ppm_face_interpolant_exact_for_cubic_cell_averages(oracle_mod):
    # For cell averages of a cubic, the unlimited fourth-order face interpolant is
    # exact; with a gentle monotone cubic neither limiter is active.
    P = lambda x: 2.0 + 0.5 * x + 0.01 * x ** 2 + 0.0002 * x ** 3
    Pint = lambda x: 2.0 * x + 0.25 * x ** 2 + 0.01 / 3 * x ** 3 + 0.00005 * x ** 4
    q = np.array([Pint(c + 0.5) - Pint(c - 0.5) for c in range(14)])
    aL, aR = oracle_mod.ppm_pencil(q)
    for c in range(2, 12):
        assert aL[c] == pytest.approx(P(c - 0.5), rel=2e-15)
        assert aR[c] == pytest.approx(P(c + 0.5), rel=2e-15)


def test_ppm_keeps_a_step_sharp(oracle_mod):
    q = np.where(np.arange(14) <= 6, 0.0, 1.0)
    aL, aR = oracle_mod.ppm_pencil(q)
    for c in range(2, 12):
        assert aL[c] == q[c] and aR[c] == q[c]


def test_ppm_flattens_a_local_extremum(oracle_mod):
    q = np.array([0, 0.1, 0.2, 0.3, 0.4, 0.5, 1.0, 0.5, 0.4, 0.3, 0.2, 0.1, 0, 0])
    aL, aR = oracle_mod.ppm_pencil(q)
    assert aL[6] == 1.0 and aR[6] == 1.0


@pytest.mark.parametrize("seed", range(5))
def test_ppm_limited_parabola_is_monotone(oracle_mod, seed):
    # CW84: after limiting, either the cell is flat, or the parabola through
    # (aL, a, aR) has no interior extremum: |6(a - (aL+aR)/2)| <= |aR - aL|,
    # with equality exactly when one face was pulled in (extremum on the edge).
    rng = np.random.default_rng(seed)
    q = np.cumsum(rng.normal(0, 1, 14)) + rng.normal(0, 0.3, 14)
    aL, aR = oracle_mod.ppm_pencil(q)
    for c in range(2, 12):
        a, l, r = q[c], aL[c], aR[c]
        if l == a and r == a:
            continue
        assert (r - a) * (a - l) > 0
        a6 = 6.0 * (a - 0.5 * (l + r))
        assert abs(a6) <= abs(r - l) * (1 + 1e-12)
        # face values lie within the range of the neighbouring cell values
        lo = min(q[c - 1], q[c], q[c + 1])
        hi = max(q[c - 1], q[c], q[c + 1])
        assert lo - 1e-12 <= l <= hi + 1e-12 and lo - 1e-12 <= r <= hi + 1e-12


# ---------------------------------------------------------------------------
# face EOS and numerical flux
# ---------------------------------------------------------------------------

def cons(rho, v, p, X=(0.1, 0.2, 0.3, 0.4, 0.5)):
    return np.array(W.conserved_from_primitive(rho, v[0], v[1], v[2], p, list(X)), float)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("form", [0, 1])
def test_flux_of_a_uniform_state_is_the_physical_flux(oracle_mod, d, form):
    rho, v, p = 1.3, np.array([0.4, -0.7, 0.25]), 0.9
    U = cons(rho, v, p)
    F, a = oracle_mod.face_flux(U, U, d, form=form)
    u = v[d]
    E = p / (G53 - 1) + 0.5 * rho * (v @ v)
    expect = U * u
    expect[1 + d] = rho * v[d] * u + p
    expect[4] = (E + p) * u
    np.testing.assert_allclose(F, expect, rtol=1e-14, atol=1e-15)
    assert a == pytest.approx(abs(u) + math.sqrt(G53 * p / rho), rel=1e-15)


def test_central_upwind_equals_central_for_symmetric_speeds(oracle_mod):
    # u_L = u_R = 0 and c_L = c_R (rho and p both doubled) give a+ = -a- = c.
    UL = cons(1.0, (0, 0.0, 0.0), 1.0, (0.1, 0.2, 0.3, 0.4, 0.5))
    UR = cons(2.0, (0, 0.0, 0.0), 2.0, (0.9, 0.8, 0.7, 0.6, 0.5))
    F0, a0 = oracle_mod.face_flux(UL, UR, 0, form=0)
    F1, a1 = oracle_mod.face_flux(UL, UR, 0, form=1)
    assert a0 == a1
    assert np.array_equal(F0, F1)


def test_central_flux_is_rusanov_form(oracle_mod):
    UL = cons(1.0, (0.3, 0.1, 0.0), 1.0)
    UR = cons(0.2, (-0.2, 0.0, 0.4), 0.3)
    F, a = oracle_mod.face_flux(UL, UR, 0, form=1)

    def phys(U):
        rho, s, E = U[0], U[1:4], U[4]
        u = s[0] / rho
        p = (G53 - 1) * (E - 0.5 * (s @ s) / rho)
        out = U * u
        out[1] += p
        out[4] = (E + p) * u
        return out, abs(u) + math.sqrt(G53 * p / rho)
    FL, aL = phys(UL)
    FR, aR = phys(UR)
    amax = max(aL, aR)
    np.testing.assert_allclose(F, 0.5 * (FL + FR) - 0.5 * amax * (UR - UL), rtol=1e-13, atol=1e-15)
    assert a == pytest.approx(amax, rel=1e-15)


def test_supersonic_face_takes_the_upwind_flux(oracle_mod):
    UL = cons(1.0, (5.0, 0.2, 0.0), 1.0)
    UR = cons(0.8, (4.0, 0.0, 0.1), 0.7)
    F, _ = oracle_mod.face_flux(UL, UR, 0, form=0)
    FL, _ = oracle_mod.face_flux(UL, UL, 0, form=0)
    np.testing.assert_allclose(F, FL, rtol=1e-14)
    Fm, _ = oracle_mod.face_flux(UR * np.array([1, -1, 1, 1, 1, 1, 1, 1, 1, 1, 1]),
                                 UL * np.array([1, -1, 1, 1, 1, 1, 1, 1, 1, 1, 1]), 0, form=0)
    FRm, _ = oracle_mod.face_flux(UL * np.array([1, -1, 1, 1, 1, 1, 1, 1, 1, 1, 1]),
                                  UL * np.array([1, -1, 1, 1, 1, 1, 1, 1, 1, 1, 1]), 0, form=0)
    np.testing.assert_allclose(Fm, FRm, rtol=1e-14)


def test_dual_energy_switch(oracle_mod):
    rho, p = 1e-6, 1e-12
    v = np.array([3.0, 0.0, 0.0])          # e_i / E ~ 1e-7 < eta: tracer used
    U = cons(rho, v, p)
    U[5] = 2.0e-8                          # tau inconsistent on purpose
    u, pf, c = oracle_mod.face_eos(U, 0)
    assert u == pytest.approx(3.0, rel=1e-15)
    assert pf == pytest.approx((G53 - 1) * 2.0e-8 ** G53, rel=1e-14)
    assert c == pytest.approx(math.sqrt(G53 * pf / rho), rel=1e-14)
    U2 = cons(1.0, (0.1, 0.0, 0.0), 1.0)
    U2[5] = 123.0                          # tracer ignored when e_i is large
    _, p2, _ = oracle_mod.face_eos(U2, 0)
    assert p2 == pytest.approx(1.0, rel=1e-14)
    _, p3, _ = oracle_mod.face_eos(U, 0, eta=0.0)   # switch disabled
    assert p3 == pytest.approx((G53 - 1) * (U[4] - 0.5 * rho * 9.0), rel=1e-6)


# ---------------------------------------------------------------------------
# whole-stage invariants
# ---------------------------------------------------------------------------

NB = (2, 2, 2)


def _grid(nb=NB, dx=1.0 / 16):
    return W.uniform_grid(nb, (0.0, 0.0, 0.0), dx)


def _step(oracle_mod, G, nb=NB, dt=0.004, stages=3, form=0):
    g = _grid(nb)
    o = oracle_mod.Oracle(g, flux_form=form)
    U = o.fill_ghosts(H.scatter(G, nb))
    if stages == 1:
        U1, ms, st = o.stage(U, dt)
    else:
        U1, ms, st = o.rk3_step(U, dt)
    assert st == 0
    return H.gather(U1, nb), ms


@pytest.mark.parametrize("form", [0, 1])
def test_uniform_state_is_preserved_bit_exactly(oracle_mod, form):
    rng = np.random.default_rng(7)
    for _ in range(3):
        rho, p = rng.uniform(0.1, 3), rng.uniform(0.1, 3)
        v = rng.uniform(-1, 1, 3)
        X = rng.uniform(0, 1, 5)
        G = H.prim_to_global(*(np.full((16, 16, 16), x) for x in (rho, *v, p)), [np.full((16, 16, 16), x) for x in X])
        out, ms = _step(oracle_mod, G, form=form)
        assert np.array_equal(out, G)
        assert ms[0] == pytest.approx(np.max(np.abs(v)) + math.sqrt(G53 * p / rho), rel=1e-14)
        assert ms[1] == pytest.approx(ms[0] * 16, rel=1e-15)


def test_conservation_on_a_periodic_domain(oracle_mod):
    G = H.random_smooth_global((16, 16, 16), 11)
    g = _grid()
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts(H.scatter(G, NB))
    U1, _, st = o.rk3_step(U, 0.01)
    assert st == 0
    for f in range(W.NF):
        before, absb = H.exact_total(g, U, f)
        after, _ = H.exact_total(g, U1, f)
        assert abs(after - before) <= 1e-13 * absb, (f, after - before, absb)
    # the state did change
    assert np.max(np.abs(U1 - U)[:, :, 3:11, 3:11, 3:11]) > 1e-3


def _mirror(G, axis):
    """Reflect the global state along axis (0=x,1=y,2=z) on the periodic domain."""
    ax = 3 - axis  # array axes: [f, z, y, x]
    M = np.flip(G, axis=ax).copy()
    M[1 + axis] *= -1.0
    return M


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_is_bit_exact(oracle_mod, axis):
    G = H.random_smooth_global((16, 16, 16), 21 + axis)
    out, _ = _step(oracle_mod, G)
    outm, _ = _step(oracle_mod, _mirror(G, axis))
    assert np.array_equal(_mirror(out, axis), outm)


def _swap(G, a, b):
    axes = {0: 3, 1: 2, 2: 1}
    M = np.swapaxes(G, axes[a], axes[b]).copy()
    M[[1 + a, 1 + b]] = M[[1 + b, 1 + a]]
    return M


def test_axis_permutation_symmetry(oracle_mod):
    G = H.random_smooth_global((16, 16, 16), 31)
    out, _ = _step(oracle_mod, G)
    # x<->y: every sum involved is commutative, so the result is bit-exact
    outxy, _ = _step(oracle_mod, _swap(G, 0, 1))
    assert np.array_equal(_swap(out, 0, 1), outxy)
    # x<->z reorders a non-associative sum: equal to round-off
    outxz, _ = _step(oracle_mod, _swap(G, 0, 2))
    scale = np.max(np.abs(out), axis=(1, 2, 3))[:, None, None, None]
    assert np.max(np.abs(_swap(out, 0, 2) - outxz) / scale) < 1e-14


@pytest.mark.parametrize("shift", [3, 8])
def test_translation_across_subgrid_seams_is_bit_exact(oracle_mod, shift):
    G = H.random_smooth_global((16, 16, 16), 41)
    out, _ = _step(oracle_mod, G)
    outs, _ = _step(oracle_mod, np.roll(G, shift, axis=3))
    assert np.array_equal(np.roll(out, shift, axis=3), outs)


def test_one_dimensional_data_gives_identical_rows(oracle_mod):
    x = (np.arange(16) + 0.5) / 16
    rho = np.broadcast_to(1.0 + 0.5 * (x > 0.5), (16, 16, 16))
    p = np.broadcast_to(1.0 + 0.2 * np.sin(2 * np.pi * x), (16, 16, 16))
    vx = np.broadcast_to(0.3 * np.cos(2 * np.pi * x), (16, 16, 16))
    z = np.zeros((16, 16, 16))
    G = H.prim_to_global(rho, vx, z, z, p)
    out, _ = _step(oracle_mod, G)
    for f in range(W.NF):
        assert np.all(out[f] == out[f][0:1, 0:1, :])
    assert np.all(out[2] == 0.0) and np.all(out[3] == 0.0)


def test_nonfinite_and_nonpositive_density_are_reported(oracle_mod):
    G = H.random_smooth_global((16, 16, 16), 51)
    g = _grid()
    o = oracle_mod.Oracle(g)
    U = o.fill_ghosts(H.scatter(G, NB))
    U[3, 2, 5, 5, 5] = np.nan
    _, _, st = o.stage(U, 0.001)
    assert st == -4
    U = o.fill_ghosts(H.scatter(G, NB))
    U[1, 0, 4, 4, 4] = -1.0
    _, _, st = o.stage(U, 0.001)
    assert st == -4


# ---------------------------------------------------------------------------
# accuracy: exact Riemann solution and convergence order
# ---------------------------------------------------------------------------

def _load_golden(name):
    vals = {}
    for line in open(__file__.replace("test_oracle_pins.py", "golden/" + name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_exact_riemann_solver_matches_textbook():
    gold = _load_golden("sod_toro_test1.txt")
    p, u, rl, rr = R.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gold["gamma"])
    assert p == pytest.approx(gold["p_star"], abs=1e-5)
    assert u == pytest.approx(gold["u_star"], abs=1e-5)
    assert rl == pytest.approx(gold["rho_star_L"], abs=1e-5)
    assert rr == pytest.approx(gold["rho_star_R"], abs=1e-5)


@functools.lru_cache(maxsize=None)
def _sod_1d(oracle_mod, ncell, t_end=0.2):
    nsub = ncell // 8
    dx = 1.0 / ncell
    g = H.quasi_1d_grid(nsub, dx, periodic_x=False)
    x = (np.arange(ncell) + 0.5) * dx
    left = x < 0.5
    sh = (8, 8, ncell)
    rho = np.broadcast_to(np.where(left, 1.0, 0.125), sh)
    p = np.broadcast_to(np.where(left, 1.0, 0.1), sh)
    z = np.zeros(sh)
    G = H.prim_to_global(rho, z, z, z, p)
    o = oracle_mod.Oracle(g)
    U, t, n = H.advance(o, H.scatter(G, (nsub, 1, 1)), t_end, 0.4)
    out = H.gather(U, (nsub, 1, 1))
    rho_num = out[0, 4, 4, :]
    rho_ex, _, _ = R.sample((x - 0.5) / t, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, G53)
    return np.sum(np.abs(rho_num - rho_ex)) * dx, out


def test_sod_tube_converges_to_exact_solution(oracle_mod):
    # calibrated once: L1(rho) = 5.52e-3, 2.75e-3, 1.35e-3 (first order, as
    # expected at a shock and a contact); gates frozen just above
    errs = [_sod_1d(oracle_mod, n)[0] for n in (128, 256, 512)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[2] <= 1.5e-3, errs
    assert min(orders) >= 0.95, (errs, orders)


def test_sod_star_state_plateau(oracle_mod):
    # in the middle of the star region between contact and shock the density
    # plateau equals the exact rho*_R, pressure p* (to the scheme's accuracy)
    _, out = _sod_1d(oracle_mod, 512)
    p_star, u_star, _, rr = R.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, G53)
    S = R.shock_speed(0.125, 0.0, 0.1, p_star, G53)
    xm = 0.5 + 0.2 * 0.5 * (u_star + S)
    i = int(xm * 512)
    rho = out[0, 4, 4, i]
    vx = out[1, 4, 4, i] / rho
    assert rho == pytest.approx(rr, rel=5e-3)
    assert vx == pytest.approx(u_star, rel=5e-3)


def _advected_wave_error(oracle_mod, ncell):
    nsub = ncell // 8
    dx = 1.0 / ncell
    g = H.quasi_1d_grid(nsub, dx, periodic_x=True)
    xl = np.arange(ncell) * dx
    # exact cell averages of rho = 1 + 0.2 sin(2 pi x)
    avg = 1.0 + 0.2 * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * (xl + dx))) / (2 * np.pi * dx)
    sh = (8, 8, ncell)
    rho = np.broadcast_to(avg, sh)
    one = np.ones(sh)
    z = np.zeros(sh)
    G = H.prim_to_global(rho, one, z, z, one)
    o = oracle_mod.Oracle(g)
    U, t, n = H.advance(o, H.scatter(G, (nsub, 1, 1)), 1.0, 0.4)
    out = H.gather(U, (nsub, 1, 1))
    return np.sum(np.abs(out[0, 4, 4, :] - avg)) * dx


def test_smooth_advected_wave_convergence_order(oracle_mod):
    # calibrated once: L1 = 1.31e-2, 3.30e-3, 8.56e-4, 2.32e-4, orders 1.98,
    # 1.95, 1.88 (limiter clipping at the extrema keeps it below 3)
    errs = [_advected_wave_error(oracle_mod, n) for n in (16, 32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert orders[-1] >= 1.8, (errs, orders)
    assert errs[-1] <= 2.5e-4, errs


# ---------------------------------------------------------------------------
# ghost fill geometry (uniform, outflow, AMR) and totals
# ---------------------------------------------------------------------------

def _linear(x, y, z):
    return 0.7 + 1.3 * x - 0.4 * y + 2.1 * z


def _ghost_center(grid, s, face, layer, c1, c2):
    a = W.FACE_AXIS[face]
    side = W.FACE_SIDE[face]
    b1, b2 = W.TRANSVERSE[a]
    idx = [0, 0, 0]
    idx[a] = W.NX + layer if side else -1 - layer
    idx[b1], idx[b2] = c1, c2
    return grid.origin[s] + (np.array(idx) + 0.5) * grid.dx[s], idx


def test_amr_ghost_fill_geometry(oracle_mod):
    w = W.config(3)
    g = w.grid
    U = W.empty_state(g.n)
    x, y, z = g.cell_centers()
    for f in range(W.NF):
        U[:, f, 3:11, 3:11, 3:11] = _linear(x, y, z) + f
    o = oracle_mod.Oracle(g)
    o.fill_ghosts(U)
    rng = np.random.default_rng(3)
    checked = {-1: 0, 0: 0, 1: 0, "out": 0}
    for s in rng.choice(g.n, 400, replace=False):
        for face in range(6):
            rel = g.neighbor_rel[s, face]
            nb0 = g.neighbor[s, face, 0]
            for layer in range(3):
                for c1 in (0, 3, 5, 7):
                    for c2 in (1, 4, 6):
                        pc, idx = _ghost_center(g, s, face, layer, c1, c2)
                        val = U[s, 2, idx[2] + 3, idx[1] + 3, idx[0] + 3]
                        if nb0 < 0:
                            a = W.FACE_AXIS[face]
                            jdx = list(idx)
                            jdx[a] = 7 if W.FACE_SIDE[face] else 0
                            expect = U[s, 2, jdx[2] + 3, jdx[1] + 3, jdx[0] + 3]
                            checked["out"] += 1
                        elif rel == -1:
                            # centre of the coarse cell that contains the ghost centre
                            h = g.dx[nb0]
                            ci = np.floor((pc - g.origin[nb0]) / h)
                            assert np.all(ci >= 0) and np.all(ci < 8)
                            expect = _linear(*(g.origin[nb0] + (ci + 0.5) * h)) + 2
                        else:
                            # same level, or mean of 8 fine centres = the coarse centre
                            expect = _linear(*pc) + 2
                        checked[rel if nb0 >= 0 else "out"] += nb0 >= 0
                        assert val == pytest.approx(expect, rel=1e-14, abs=1e-13), (s, face, rel, layer, c1, c2)
    assert all(v > 0 for v in checked.values()), checked


def test_totals_match_exact_sum(oracle_mod):
    w = W.config(3)
    U = w.state()
    o = oracle_mod.Oracle(w.grid)
    t = o.totals(U)
    for f in range(W.NF):
        ex, ab = H.exact_total(w.grid, U, f)
        assert abs(t[f] - ex) <= 1e-15 * ab + 1e-300


# ---------------------------------------------------------------------------
# diagnostics (Section V-B.1: total mass, angular momentum, centre of mass of
# each star), pinned by closed forms and by an identity between its outputs
# ---------------------------------------------------------------------------

def _box_state(nb, lo, h, fill):
    """Padded state on a uniform non-periodic grid from fill(x, y, z) -> list of 11 global fields."""
    g = W.uniform_grid(nb, lo, h, periodic=(False, False, False))
    N = [n * W.NX for n in nb]
    c = [lo[a] + (np.arange(N[a]) + 0.5) * h for a in range(3)]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    G = np.stack(fill(x, y, z))
    return g, H.scatter(G, nb)


def test_diagnostics_solid_body_rotation_closed_form(oracle_mod):
    """Uniform density rho0 rotating about z at omega in the cube [-a, a]^3:
    Lz = rho0 omega sum (x_c^2 + y_c^2) h^3, and the midpoint rule for x^2 is
    exact up to its known error: sum_i x_i^2 h = 2a^3/3 - a h^2/6 per axis."""
    a, nbs = 1.0, 4
    N = nbs * W.NX
    h = 2 * a / N
    rho0, om = 1.7, 0.3
    zero = lambda x: np.zeros_like(x)

    def fill(x, y, z):
        rho = np.full_like(x, rho0)
        return [rho, -rho0 * om * y, rho0 * om * x, zero(x), rho, rho, rho, zero(x), zero(x), zero(x), zero(x)]

    g, U = _box_state((nbs, nbs, nbs), (-a, -a, -a), h, fill)
    d = oracle_mod.Oracle(g).diagnostics(U)
    sum_x2 = (2 * a) ** 2 * (2 * a ** 3 / 3 - a * h ** 2 / 6)   # sum over cells of x_c^2 h^3
    Lz = rho0 * om * 2 * sum_x2
    assert abs(d[3] - Lz) <= 1e-13 * Lz
    assert abs(d[1]) <= 1e-14 * Lz and abs(d[2]) <= 1e-14 * Lz
    assert abs(d[0] - rho0 * (2 * a) ** 3) <= 1e-13 * rho0 * (2 * a) ** 3
    assert np.all(np.abs(d[5:8]) <= 1e-14)          # star 1 spread over the whole cube: centre 0
    assert d[8] == 0.0 and np.all(d[9:12] == 0.0)   # no star 2


def test_diagnostics_centre_of_symmetric_ball(oracle_mod):
    """Star 1 material in a ball whose centre c is a cell corner, star 2 in
    another: by symmetry each centre of mass is its ball's centre, each mass
    the sum over the cells inside the ball."""
    h = 1.0 / 16
    c1, c2, R = np.array([0.25, -0.125, 0.5]), np.array([-0.375, 0.25, -0.25]), 0.3
    zero = lambda x: np.zeros_like(x)

    def fill(x, y, z):
        in1 = ((x - c1[0]) ** 2 + (y - c1[1]) ** 2 + (z - c1[2]) ** 2 < R * R).astype(float)
        in2 = ((x - c2[0]) ** 2 + (y - c2[1]) ** 2 + (z - c2[2]) ** 2 < R * R).astype(float)
        rho = 0.1 + 2.0 * in1 + 3.0 * in2
        return [rho, zero(x), zero(x), zero(x), rho, rho, 2.0 * in1, 3.0 * in2, zero(x), zero(x), zero(x)]

    g, U = _box_state((4, 4, 4), (-1.0, -1.0, -1.0), h, fill)
    d = oracle_mod.Oracle(g).diagnostics(U)
    assert np.all(np.abs(d[5:8] - c1) <= 1e-14) and np.all(np.abs(d[9:12] - c2) <= 1e-14)
    n1 = d[4] / (2.0 * h ** 3)
    assert abs(n1 - round(n1)) <= 1e-9 and round(n1) > 100    # a whole number of cells
    assert abs(d[8] / (3.0 * h ** 3) - round(n1)) <= 1e-9      # congruent balls


def test_diagnostics_translation_identity(oracle_mod):
    """For s = rho v with uniform v and star 1 = all the mass, the angular
    momentum about the origin is M (R1 x v): pins the signs and indices of the
    cross product against the first moments, on the AMR octree."""
    w = W.config(3)
    U = w.state()
    v = np.array([0.3, -0.7, 1.1])
    U[:, 1:4] = U[:, 0:1] * v[None, :, None, None, None]
    U[:, 6] = U[:, 0]
    d = oracle_mod.Oracle(w.grid).diagnostics(U)
    expect = d[4] * np.cross(d[5:8], v)
    scale = d[0] * np.abs(v).max() * 2.0
    assert np.all(np.abs(d[1:4] - expect) <= 1e-13 * scale), (d[1:4], expect)
    assert abs(d[4] - d[0]) <= 1e-14 * d[0]


# ---------------------------------------------------------------------------
# coarse-fine flux correction (Section V-B.1: compute_fluxes corrects the
# fluxes on coarse-fine boundaries): the AMR step then conserves to round-off
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("reflux", [True, False])
def test_amr_conservation_needs_flux_correction(oracle_mod, reflux):
    g, U = H.amr_blob_state()
    assert np.any(g.neighbor_rel == 1)             # the grid has coarse-fine faces
    o = oracle_mod.Oracle(g, reflux=reflux)
    o.fill_ghosts(U)
    _, ms, st = o.stage(U, 0.0)
    assert st == 0
    dt = 0.4 / ms[1]
    V, _, st = o.rk3_step(U, dt)
    assert st == 0
    drift = []
    for f in (0, 4, 5, 6, 7, 8):                   # mass, energy, tau, scalars: no boundary flux
        b, ab = H.exact_total(g, U, f)
        a, _ = H.exact_total(g, V, f)
        drift.append(abs(a - b) / ab)
    if reflux:
        assert max(drift) <= 1e-14, drift
    else:
        assert max(drift) > 1e-9, drift             # without the correction the AMR step leaks


# ---------------------------------------------------------------------------
# Dual-energy resynchronisation of the entropy tracer
# ---------------------------------------------------------------------------

def test_tau_resync_tracer_pressure_matches_energy_pressure(oracle_mod):
    # What the reset is for: afterwards the face EOS gives the same pressure
    # whether it takes the internal energy from the total energy (switch off)
    # or from the tracer (switch forced on), in every cell the switch trusts;
    # cells below the switch keep their tracer bit for bit.
    grid, U, cold = H.resync_case()
    o = oracle_mod.Oracle(grid)
    V = U.copy()
    n_reset = o.tau_resync(V)
    inner = (slice(None), slice(3, 11), slice(3, 11), slice(3, 11))
    cold_in = cold[inner[0], inner[1], inner[2], inner[3]]
    assert n_reset == int((~cold_in).sum()) == 8 * 512 - 16 * 16 * 4
    Vi = V[:, :, 3:11, 3:11, 3:11]
    Ui = U[:, :, 3:11, 3:11, 3:11]
    assert np.array_equal(Vi[:, 5][cold_in], Ui[:, 5][cold_in])
    assert not np.any(Vi[:, 5][~cold_in] == Ui[:, 5][~cold_in])
    cells = np.argwhere(~cold_in)
    worst = 0.0
    for s, k, j, i in cells[::7]:
        st = Vi[s, :, k, j, i]
        _, p_energy, _ = oracle_mod.face_eos(st, 0, G53, 0.0)
        _, p_tracer, _ = oracle_mod.face_eos(st, 0, G53, 2.0)
        worst = max(worst, abs(p_tracer - p_energy) / p_energy)
    assert worst < 1e-13


def test_tau_resync_fixed_point_of_initial_state(oracle_mod):
    # The initial conditions set tau = (p/(gamma-1))^(1/gamma) with
    # E = p/(gamma-1) + rho|v|^2/2: the tracer already matches, so the reset
    # moves it by rounding only, and touches no other field or ghost cell.
    w = W.config(3)
    U = w.state()
    o = oracle_mod.Oracle(w.grid)
    V = U.copy()
    n_reset = o.tau_resync(V)
    assert n_reset > 0.9 * w.grid.n * 512
    changed = ~((V == U) | (np.isnan(V) & np.isnan(U)))
    assert not changed[:, [0, 1, 2, 3, 4, 6, 7, 8, 9, 10]].any()
    mask = np.ones(U.shape[2:], bool)
    mask[3:11, 3:11, 3:11] = False
    assert not changed[:, :, mask].any()
    rel = np.abs(V[:, 5] - U[:, 5]) / np.abs(U[:, 5])
    assert np.nanmax(rel) < 1e-14


def test_tau_resync_idempotent_and_switch_off(oracle_mod):
    grid, U, _ = H.resync_case(seed=12)
    o = oracle_mod.Oracle(grid)
    V = U.copy()
    o.tau_resync(V)
    V2 = V.copy()
    o.tau_resync(V2)
    assert np.array_equal(V, V2, equal_nan=True)
    off = oracle_mod.Oracle(grid, de_switch=0.0)
    V3 = U.copy()
    assert off.tau_resync(V3) == 0
    assert np.array_equal(V3, U, equal_nan=True)
