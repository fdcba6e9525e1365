"""The sharded step on one GPU: two partitions of the 4096-leaf octree held in
one process, each advanced by its own handle on its local grid (owned
sub-grids, then proxy slots).  Before every Shu-Osher stage the proxies get,
by device copies, only the cells their reader uses (3-layer face slabs of
same-level and coarser proxies, whole interiors of finer ones; every other
proxy cell is NaN); the finer proxies next to an owned coarse sub-grid are
listed as flux-only items, so the coarse-fine correction sees the fluxes of
remote fine neighbours; the maximum signal speed is the maximum over the two.
The gathered owned interiors after two RK3 steps equal the single-domain run
with the same library bit for bit, in both precisions (and the FP64 one is the
oracle's to 1e-12 per cell), also with the CW84 extensions, whose flattening
reads a fourth layer (4-layer slabs)."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import partition as P
from paper_2210_06437_gb300 import workloads as W
from tests import r12 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
IN = P.INTERIOR
STEPS = 2
BETA = (1.0, 0.25, 2.0 / 3.0)


@pytest.fixture(scope="module")
def hydro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build, hydro as HY
    build.build()
    return HY


def _rk3(stage, U, ms_first):
    """SSP-RK3 in Shu-Osher stages with the lagged CFL dt; stage(Uin, dt, U0, beta) -> (Uout, ms)."""
    ms = ms_first
    dts = []
    for _ in range(STEPS):
        dt = 0.4 / ms[1]
        dts.append(dt)
        U1, ms = stage(U, dt, None, BETA[0])
        U2, _ = stage(U1, dt, U, BETA[1])
        U, _ = stage(U2, dt, U, BETA[2])
    return U, dts


@pytest.mark.parametrize("cw84", [0, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sharded_step_on_one_gpu(hydro, oracle_mod, prec, cw84):
    w = W.config(3)
    grid = w.grid
    # single domain
    g = hydro.HydroGrid(grid, precision=prec)
    g.set_param(hydro.PARAM_CW84, cw84)
    depth = P.SLAB_CW84 if cw84 & 1 else P.SLAB   # flattening reads one layer further
    ids_all = torch.as_tensor(w.batches.ids, device="cuda")

    def stage1(Uin, dt, U0, beta):
        out, ms = g.step(Uin, dt, U0=U0, beta=beta, U_out=torch.empty_like(Uin), ids=ids_all,
                         batch_offsets=w.batches.offsets)
        return out, ms.cpu().numpy()

    U = torch.from_numpy(w.state()).cuda()
    _, ms0 = stage1(U, 0.0, None, 1.0)
    ref, dts_ref = _rk3(stage1, U, ms0)
    g.sync()
    ref = ref.cpu().numpy()
    g.close()
    # two partitions
    parts = [P.build(grid, r, 2) for r in range(2)]
    handles = [hydro.HydroGrid(p.local, precision=prec) for p in parts]
    for h in handles:
        h.set_param(hydro.PARAM_CW84, cw84)
    G0 = w.state()
    states = []
    for p in parts:
        UL = torch.from_numpy(P.scatter_global(p, G0)).cuda()
        UL[p.n_owned:][IN] = float("nan")
        states.append(UL)
    batch = [torch.as_tensor(np.concatenate([np.arange(p.n_owned, dtype=np.int32),
                                             P.flux_only_proxies(p) | np.int32(hydro.ITEM_FLUX_ONLY)]),
                             device="cuda") for p in parts]
    assert all(len(P.flux_only_proxies(p)) > 0 for p in parts)
    moved = []

    def stage2(Uins, dt, U0s, beta):
        moved.append(P.exchange_direct(parts, Uins, depth))
        outs, mss = [], []
        for r, p in enumerate(parts):
            out = torch.full_like(Uins[r], float("nan"))
            out, ms = handles[r].step(Uins[r], dt, U0=None if U0s is None else U0s[r], beta=beta, U_out=out,
                                      ids=batch[r])
            outs.append(out)
            mss.append(ms.cpu().numpy())
        return outs, np.maximum(mss[0], mss[1])

    _, ms0s = stage2(states, 0.0, None, 1.0)
    assert np.array_equal(ms0s, ms0)
    outs, dts = _rk3(stage2, states, ms0s)
    for h in handles:
        h.sync()
    assert dts == dts_ref
    got = np.concatenate([outs[r][:p.n_owned].cpu().numpy() for r, p in enumerate(parts)])
    assert np.array_equal(got[IN], ref[IN])
    # the slabs moved fewer bytes than whole interiors would
    whole = sum(len(p.proxies) for p in parts) * 11 * 512 * 8
    assert max(moved) < (0.7 if depth == P.SLAB else 0.8) * whole
    if prec == "fp64":   # and the FP64 run is the oracle's, to the pow of the dual-energy switch
        o = oracle_mod.Oracle(grid, cw84=cw84)
        Uo = w.state()
        o.fill_ghosts(Uo)
        for dt in dts_ref:
            Uo, _, st = o.rk3_step(Uo, dt)
        res = R.r12(got, Uo)
        assert np.all(res["err"] <= 1e-12), R.summary(res)
    for h in handles:
        h.close()
