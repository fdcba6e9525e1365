"""GPU parity of the three-dimensional reconstruction with Simpson face
quadrature (HYDRO_PARAM_RECON3D, grids of one level, both precisions) against
the oracle's `stage3d` / `rk3_step3d`, through the C ABI.

Gate: the FP64 gate of the other parity tests (R12 <= 1e-12 per field; the
kernels round every operation as the oracle does, so the results agree bit for
bit except where the dual-energy switch evaluates pow), the max speeds to
1e-14.  The GPU input keeps NaN ghost canaries: the face-average kernel reads
face, edge and corner neighbours' interiors and never a ghost cell.  Cases:
the periodic Sod tube and lognormal box (one stage with the Shu-Osher blend,
one RK3 step), a 3 x 2 x 2 box with outflow boundaries (edge and corner cells
clamped at the domain boundary, unequal sub-grid counts per axis), a uniform
state, the parameter's refusals, and bit identity with the oracle for both
flux forms with and without the dual-energy switch.  Mixed precision (FP32
reconstruction and fluxes, FP64 update) against the same oracle at the mixed
gate (R12 <= 1e-5), outside the margin cells of the transverse tests."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import r12 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
IN = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))


@pytest.fixture(scope="module")
def hydro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build, hydro as HY
    build.build()
    return HY


def _grid3d(hydro, grid):
    g = hydro.HydroGrid(grid, precision="fp64")
    g.set_param(hydro.PARAM_RECON3D, 1)
    return g


def _check(got, ref):
    res = R.r12(got, ref)
    assert np.all(res["err"] <= TOL), R.summary(res)
    return res


def _box(outflow_nb=(3, 2, 2), seed=5):
    nb = outflow_nb
    g = W.uniform_grid(nb, (0.0, 0.0, 0.0), 1.0 / (8 * max(nb)), periodic=(False, False, False))
    G = H.random_smooth_global((8 * nb[2], 8 * nb[1], 8 * nb[0]), seed)
    return g, H.scatter(G, nb)


def _cases():
    return ["sod16", "lognormal64", "outflow_box"]


def _workload(name):
    if name == "outflow_box":
        return _box()
    w = W.config(1 if name == "sod16" else 2)
    return w.grid, w.state()


@pytest.mark.parametrize("name", _cases())
def test_stage_matches_oracle(hydro, oracle_mod, name):
    grid, U = _workload(name)
    o = oracle_mod.Oracle(grid)
    Uf = o.fill_ghosts_full(U.copy())
    _, ms0, st = o.stage3d(Uf, 0.0)
    assert st == 0
    dt = 0.4 / ms0[1]
    U0 = Uf.copy()
    U0[IN] *= 1.0 + 1e-3 * np.sin(np.arange(U0[IN].size).reshape(U0[IN].shape))
    ref, ms_o, st = o.stage3d(Uf, dt, U0=U0, beta=0.25)
    assert st == 0
    g = _grid3d(hydro, grid)
    Ud, U0d = torch.from_numpy(U).cuda(), torch.from_numpy(U0).cuda()
    out = Ud.clone()
    out, ms = g.step(Ud, dt, U0=U0d, beta=0.25, U_out=out)
    g.sync()
    got = out.cpu().numpy()
    res = _check(got, ref)
    np.testing.assert_allclose(ms.cpu().numpy(), ms_o, rtol=1e-14)
    # away from one-dimensional data (the Sod tube, where both agree) the
    # Simpson fluxes differ from the face-centre ones far beyond the parity
    # error, so the test tells the two apart
    if name != "sod16":
        mid, _, _ = o.stage(Uf, dt, U0=U0, beta=0.25)
        assert np.max(np.abs(mid[IN] - ref[IN])) > 1e3 * np.max(np.abs(got[IN] - ref[IN])) + 1e-14
    assert res["n_cells"] == grid.n * 512


@pytest.mark.parametrize("name", ["lognormal64", "outflow_box"])
def test_rk3_step_matches_oracle(hydro, oracle_mod, name):
    grid, U = _workload(name)
    o = oracle_mod.Oracle(grid)
    Uf = o.fill_ghosts_full(U.copy())
    _, ms0, _ = o.stage3d(Uf, 0.0)
    dt = 0.4 / ms0[1]
    ref, ms_o, st = o.rk3_step3d(Uf.copy(), dt)
    assert st == 0
    g = _grid3d(hydro, grid)
    Ud = torch.from_numpy(U).cuda()
    s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
    ms = g.rk3_step(Ud, dt, s1, s2)
    g.sync()
    _check(Ud.cpu().numpy(), ref)
    np.testing.assert_allclose(ms.cpu().numpy(), ms_o, rtol=1e-14)
    # a second step replays the captured graph
    ref2, _, st = o.rk3_step3d(ref.copy(), dt)
    assert st == 0
    g.rk3_step(Ud, dt, s1, s2, max_speed=ms)
    g.sync()
    _check(Ud.cpu().numpy(), ref2)


def test_uniform_state_is_kept_bit_exact(hydro):
    grid, _ = _box()
    G = H.prim_to_global(*(np.full((16, 16, 24), v) for v in (1.3, 0.2, -0.4, 0.1, 0.8)))
    U = H.scatter(G, (3, 2, 2))
    g = _grid3d(hydro, grid)
    Ud = torch.from_numpy(U).cuda()
    out, _ = g.step(Ud, 1e-3, U_out=Ud.clone())
    g.sync()
    assert np.array_equal(out.cpu().numpy()[IN], U[IN])


def test_parameter_refusals(hydro):
    w1, w3 = W.config(1), W.config(3)
    g = hydro.HydroGrid(w3.grid, precision="mixed")
    with pytest.raises(hydro.HydroError):
        g.set_param(hydro.PARAM_RECON3D, 1)
    g = hydro.HydroGrid(w3.grid, precision="fp64")
    with pytest.raises(hydro.HydroError):
        g.set_param(hydro.PARAM_RECON3D, 1)
    g = hydro.HydroGrid(w1.grid, precision="fp64")
    g.set_param(hydro.PARAM_CW84, 1)
    with pytest.raises(hydro.HydroError):
        g.set_param(hydro.PARAM_RECON3D, 1)
    g.set_param(hydro.PARAM_CW84, 0)
    g.set_param(hydro.PARAM_RECON3D, 1)
    with pytest.raises(hydro.HydroError):
        g.set_param(hydro.PARAM_CW84, 1)
    with pytest.raises(hydro.HydroError):
        g.set_param(hydro.PARAM_RECON3D, 2)
    g.set_param(hydro.PARAM_RECON3D, 0)


@pytest.mark.parametrize("form,de_switch", [(0, 1e-3), (1, 1e-3), (0, 0.0)])
@pytest.mark.parametrize("name", _cases())
def test_bit_identical_to_oracle(hydro, oracle_mod, name, form, de_switch):
    """Every operation rounds as the oracle's does, so one blended stage, its
    maximum speeds and one RK3 step agree bit for bit (these states never take
    the dual-energy branch, whose pow neither side rounds correctly)."""
    grid, U = _workload(name)
    o = oracle_mod.Oracle(grid, flux_form=form, de_switch=de_switch)
    Uf = o.fill_ghosts_full(U.copy())
    _, ms0, _ = o.stage3d(Uf, 0.0)
    dt = 0.4 / ms0[1]
    U0 = Uf.copy()
    U0[IN] *= 1.0 + 1e-3 * np.cos(np.arange(U0[IN].size).reshape(U0[IN].shape))
    ref, ms_o, st = o.stage3d(Uf, dt, U0=U0, beta=2.0 / 3.0)
    assert st == 0
    g = hydro.HydroGrid(grid, precision="fp64", flux_form=form, de_switch=de_switch)
    g.set_param(hydro.PARAM_RECON3D, 1)
    out, ms = g.step(torch.from_numpy(U).cuda(), dt, U0=torch.from_numpy(U0).cuda(), beta=2.0 / 3.0,
                     U_out=torch.from_numpy(U).cuda())
    g.sync()
    assert np.array_equal(out.cpu().numpy()[IN], ref[IN])
    assert np.array_equal(ms.cpu().numpy(), ms_o)
    ref3, _, st = o.rk3_step3d(Uf.copy(), dt)
    assert st == 0
    Ud = torch.from_numpy(U).cuda()
    g.rk3_step(Ud, dt, torch.empty_like(Ud), torch.empty_like(Ud))
    g.sync()
    assert np.array_equal(Ud.cpu().numpy()[IN], ref3[IN])


NONMOM = [0, 4, 5, 6, 7, 8, 9, 10]
MIXED_TOL = 1e-5
# One RK3 step on the lognormal box, whose passive scalars are random from cell
# to cell: measured 2.0e-5 in one cell of 262,144 outside the margin cells
# (ρX3; every other gated value <= 3.6e-6).  The oracle itself, fed its own
# stage inputs rounded to FP32 (FP64 arithmetic otherwise), departs from the
# exact step by up to 2.2e-5 per cell: the size is the scheme's sensitivity to
# its inputs on this data over three stages, not the kernels' FP32 arithmetic.
# The single stage meets 1e-5 (measured 4.6e-7).
MIXED_RK3_GATE = {"lognormal64": 5e-5}


def _check_mixed(got, ref, margin, gate=MIXED_TOL):
    """The mixed gate of the other parity tests: R12 <= 1e-5 on the
    non-momentum fields and the momenta against max(|s|, rho c), outside the
    margin cells (here the faces whose transverse tests or dual-energy test
    sit within 64 x 2^-24 of their thresholds, which FP32 may take the other
    way: a parabola against a constant or a line)."""
    res = R.r12(got, ref, margin)
    assert np.all(res["err"][NONMOM] <= gate), R.summary(res)
    mom = R.momentum_scaled(got, ref, margin=margin)
    assert np.all(mom <= gate), (mom, R.summary(res))
    return res


@pytest.mark.parametrize("name", _cases())
def test_mixed_stage_and_rk3_match_oracle(hydro, oracle_mod, name):
    """Mixed precision (FP32 reconstruction, transverse parabolas, point
    fluxes and Simpson sums; FP64 update): one blended stage and one RK3 step
    (Shu-Osher stages) against the FP64 oracle."""
    grid, U = _workload(name)
    o = oracle_mod.Oracle(grid)
    eps = R.EPS["mixed"]
    Uf = o.fill_ghosts_full(U.copy())
    _, ms0, _ = o.stage3d(Uf, 0.0)
    dt = 0.4 / ms0[1]
    U0 = Uf.copy()
    U0[IN] *= 1.0 + 1e-3 * np.sin(np.arange(U0[IN].size).reshape(U0[IN].shape))
    ref, ms_o, st = o.stage3d(Uf, dt, U0=U0, beta=0.25)
    assert st == 0
    g = hydro.HydroGrid(grid, precision="mixed")
    g.set_param(hydro.PARAM_RECON3D, 1)
    Ud = torch.from_numpy(U).cuda()
    out, ms = g.step(Ud, dt, U0=torch.from_numpy(U0).cuda(), beta=0.25, U_out=Ud.clone())
    g.sync()
    margin, _ = o.margin_cells3d(Uf, eps)
    _check_mixed(out.cpu().numpy(), ref, margin)
    np.testing.assert_allclose(ms.cpu().numpy(), ms_o, rtol=1e-6)
    # one RK3 step; margins over the three stage inputs
    ref3, _, st = o.rk3_step3d(Uf.copy(), dt)
    assert st == 0
    U1, _, _ = o.stage3d(Uf, dt)
    o.fill_ghosts_full(U1)
    U2, _, _ = o.stage3d(U1, dt, U0=Uf, beta=0.25)
    margin3 = None
    for S in (Uf, U1, U2):
        margin3, _ = o.margin_cells3d(S, eps, mask=margin3)
    s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
    g.rk3_step(Ud, dt, s1, s2)
    g.sync()
    res = _check_mixed(Ud.cpu().numpy(), ref3, margin3, MIXED_RK3_GATE.get(name, MIXED_TOL))
    # the margins of three stage inputs leave most cells gated (measured on
    # the oracle: 0 % of the Sod tube, 7 % of the lognormal box, 20 % of the
    # small outflow box of random smooth data)
    assert res["n_margin"] < 0.25 * res["n_cells"]


def test_mixed_shadowed_step_is_refused(hydro):
    grid, U = _box()
    g = hydro.HydroGrid(grid, precision="mixed")
    g.set_param(hydro.PARAM_RECON3D, 1)
    Ud = torch.from_numpy(U).cuda()
    S = g.empty_shadow()
    with pytest.raises(hydro.HydroError):
        g.step_shadowed(Ud, S, 1e-3)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_subset_and_empty_batches(hydro, oracle_mod, prec):
    """A batch of some sub-grids (ragged, unordered) updates exactly those, as
    the whole-grid stage does (their halos read the unlisted neighbours'
    inputs); the others keep the output buffer's contents; an empty batch
    launches nothing and reports zero speeds."""
    grid, U = _box()
    g = _grid3d_prec(hydro, grid, prec)
    Ud = torch.from_numpy(U).cuda()
    full, _ = g.step(Ud, 1e-3, U_out=torch.zeros_like(Ud))
    ids = np.array([7, 2, 11, 0, 5], np.int32)
    part, _ = g.step(Ud, 1e-3, U_out=torch.zeros_like(Ud), ids=ids)
    g.sync()
    full, part = full.cpu().numpy(), part.cpu().numpy()
    assert np.array_equal(part[ids][IN], full[ids][IN])
    rest = np.setdiff1d(np.arange(grid.n), ids)
    assert not part[rest].any()
    n0 = g.launches
    out, ms = g.step(Ud, 1e-3, U_out=torch.zeros_like(Ud), ids=np.zeros(0, np.int32))
    g.sync()
    assert g.launches == n0 and not out.any().item() and not ms.any().item()


def _grid3d_prec(hydro, grid, prec):
    g = hydro.HydroGrid(grid, precision=prec)
    g.set_param(hydro.PARAM_RECON3D, 1)
    return g


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_graph_matches_separate_steps(hydro, prec):
    """hydro_rk3_run_cfl over 3 steps (device CFL dt, totals) is bit-identical
    to 3 hydro_rk3_step_cfl calls each followed by hydro_totals."""
    w = W.config(2)
    U = w.state()
    g = _grid3d_prec(hydro, w.grid, prec)
    res = []
    for mode in ("separate", "run"):
        Ud = torch.from_numpy(U).cuda()
        s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
        ms = torch.zeros(2, dtype=torch.float64, device="cuda")
        g.step(Ud, 0.0, U_out=s1, max_speed=ms)
        dts = torch.zeros(3, dtype=torch.float64, device="cuda")
        tots = torch.zeros((3, 11), dtype=torch.float64, device="cuda")
        if mode == "separate":
            for k in range(3):
                g.rk3_step_cfl(Ud, 0.4, s1, s2, ms, dt_out=dts[k:k + 1])
                g.totals(Ud, out=tots[k])
        else:
            g.rk3_run_cfl(Ud, 0.4, s1, s2, ms, 3, dt_out=dts, totals=tots)
        g.sync()
        res.append((Ud.cpu().numpy()[IN], dts.cpu().numpy(), tots.cpu().numpy(), ms.cpu().numpy()))
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    assert np.all(res[0][1] > 0)
