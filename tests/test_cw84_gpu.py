"""GPU parity of the CW84 PPM extensions (HYDRO_PARAM_CW84: shock flattening,
contact steepening) against the oracle with the same flags, through the C ABI.
The FP64 stage evaluates them in the oracle's order and rounding, so one stage
and one RK3 step are bit-identical where the dual-energy power does not enter
(without the switch); the mixed stage meets the per-cell error (R12) of the
base scheme's tests outside cells whose flattening or steepening decision sits
near its threshold.  Cases: a periodic blast (pressure jump, converging flow:
both detectors fire), the Sod tube of configuration 1 after it has developed,
and the AMR polytrope (fourth ghost layer across coarse-fine faces, flux
correction, conservation)."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H
from tests import r12 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
IN = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))
ALL = 3


@pytest.fixture(scope="module")
def hydro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build, hydro as HY
    build.build()
    return HY


def _blast(seed=5):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(16) + 0.5,) * 3, indexing="ij")
    r2 = (x - 8) ** 2 + (y - 7.5) ** 2 + (z - 8.5) ** 2
    p = np.where(r2 < 16, 10.0, 1.0) * (1 + 0.01 * rng.standard_normal((16, 16, 16)))
    rho = np.where(r2 < 9, 2.0, 1.0) * (1 + 0.01 * rng.standard_normal((16, 16, 16)))
    v = [-0.3 * (c - 8) / 8 for c in (x, y, z)]
    return H.prim_to_global(rho, *v, p)


def _case(name, oracle_mod, de_switch):
    """(grid, padded state with ghosts filled, ids, offsets) of a test case."""
    if name == "blast":
        g = W.uniform_grid((2, 2, 2), (0.0, 0.0, 0.0), 1.0 / 16)
        U = H.scatter(_blast(), (2, 2, 2))
        ids = offs = None
    else:
        w = W.config(1 if name == "sod" else 3)
        g, U, ids, offs = w.grid, w.state(), w.batches.ids, w.batches.offsets
    o = oracle_mod.Oracle(g, de_switch=de_switch, cw84=ALL)
    o.fill_ghosts(U)
    if name == "sod":   # let the tube develop so that the shock compresses
        U, _, _ = H.advance(o, U, 0.05, 0.4)
        o.fill_ghosts(U)
    return g, U, ids, offs, o


def _run(hydro, g, U, ids, offs, prec, de_switch, cw, dt):
    h = hydro.HydroGrid(g, precision=prec, de_switch=de_switch)
    h.set_param(hydro.PARAM_CW84, cw)
    kw = {} if ids is None else {"ids": torch.as_tensor(ids, device="cuda"), "batch_offsets": offs}
    Ud = torch.from_numpy(U).cuda()
    out, ms = h.step(Ud, dt, U_out=torch.empty_like(Ud), **kw)
    V = Ud.clone()
    h.rk3_step(V, dt, torch.empty_like(V), torch.empty_like(V), **kw)
    h.sync()
    res = (out.cpu().numpy(), ms.cpu().numpy(), V.cpu().numpy())
    h.close()
    return res


@pytest.mark.parametrize("name,de_switch", [("blast", 0.0), ("sod", 0.0), ("amr", 1e-3)])
def test_fp64_matches_oracle(hydro, oracle_mod, name, de_switch):
    g, U, ids, offs, o = _case(name, oracle_mod, de_switch)
    _, ms0, _ = o.stage(U, 0.0)
    dt = 0.4 / ms0[1]
    ref1, ms_o, st = o.stage(U, dt)
    ref3, _, st3 = o.rk3_step(U, dt)
    assert st == 0 and st3 == 0
    base1 = oracle_mod.Oracle(g, de_switch=de_switch).stage(U, dt)[0]
    assert not np.array_equal(base1[IN], ref1[IN])   # the detectors fired
    one, ms, three = _run(hydro, g, U, ids, offs, "fp64", de_switch, ALL, dt)
    if de_switch == 0.0:
        assert np.array_equal(one[IN], ref1[IN])
        assert np.array_equal(ms, ms_o)
        assert np.array_equal(three[IN], ref3[IN])
    else:   # tau^gamma: pow may differ by an ulp between the two libms
        for x, r in ((one, ref1), (three, ref3)):
            res = R.r12(x, r)
            assert np.all(res["err"] <= 1e-12), R.summary(res)


# RK3-step bounds of the mixed path, from one measured run per case: cells
# above 1e-4 (non-momentum R12), their largest error, and the largest
# momentum error against rho c.  Flattening switches a coefficient on or off;
# over three stages the FP32 intermediate states (about 1e-5 from the
# oracle's) take some of those decisions the other way.
# measured: blast 0 cells, max 1.5e-7, momentum 5.7e-8; Sod 0, 2.6e-7, 5.8e-8;
# AMR polytrope 175 of 2.1 M cells (near the star's surface), max 3.6e-3,
# momentum 5.5e-2
RK3_OUTLIERS = {"blast": (0.0, 1e-5, 1e-4), "sod": (0.0, 1e-5, 1e-4), "amr": (2e-4, 5e-3, 8e-2)}


@pytest.mark.parametrize("name", ["blast", "sod", "amr"])
def test_mixed_matches_oracle(hydro, oracle_mod, name):
    """One stage: every cell but those whose flattening, steepening or
    dual-energy test sits within 64 FP32 ulps of its threshold (counted, at
    most 5 % of the cells) within the base scheme's gates.  One RK3 step: the
    measured outlier bounds above."""
    de = 1e-3
    g, U, ids, offs, o = _case(name, oracle_mod, de)
    _, ms0, _ = o.stage(U, 0.0)
    dt = 0.4 / ms0[1]
    ref1, _, _ = o.stage(U, dt)
    ref3, _, _ = o.rk3_step(U, dt)
    one, _, three = _run(hydro, g, U, ids, offs, "mixed", de, ALL, dt)
    nonmom = [f for f in range(W.NF) if f not in (1, 2, 3)]
    margin = R.margin_union(o, [U], R.EPS["mixed"])
    res = R.r12(one, ref1, margin)
    assert np.all(res["err"][nonmom] <= 1e-5), (name, R.summary(res))
    assert ((margin & R.M_CW84) != 0).sum() <= 0.05 * res["n_cells"], R.summary(res)
    gated = ((margin & R.M_SWITCH) == 0)[:, None]
    mom = R.momentum_scaled(one[IN] * gated, ref1[IN] * gated)
    assert np.all(mom <= 1e-4), (name, mom)
    e, _ = R.cell_errors(three, ref3)
    en = e[:, nonmom].max(axis=1)
    frac, emax, mmax = RK3_OUTLIERS[name]
    mom3 = R.momentum_scaled(three, ref3)
    print("CW84 mixed RK3 %s: cells above 1e-4 %d of %d, max %.2e, momentum/rho c %.2e"
          % (name, int((en > 1e-4).sum()), en.size, en.max(), mom3.max()))
    assert (en > 1e-4).sum() <= frac * en.size and en.max() <= emax, (int((en > 1e-4).sum()), float(en.max()))
    assert np.all(mom3 <= mmax), mom3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amr_conservation_with_extensions(hydro, oracle_mod, prec):
    """The extensions change the face states only: fluxes stay single-valued
    and the coarse-fine correction still conserves mass, energy and the
    scalars on the AMR blob, which nothing leaves."""
    grid, U = H.amr_blob_state()
    o = oracle_mod.Oracle(grid, cw84=ALL)
    o.fill_ghosts(U)
    _, ms0, _ = o.stage(U, 0.0)
    dt = 0.4 / ms0[1]
    _, _, three = _run(hydro, grid, U, None, None, prec, grid.de_switch, ALL, dt)
    for f in (0, 4, 5, 6, 7, 8, 9, 10):
        before, absb = H.exact_total(grid, U, f)
        after, _ = H.exact_total(grid, three, f)
        assert abs(after - before) <= 1e-13 * absb, (f, after - before, absb)
