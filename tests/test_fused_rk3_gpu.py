"""The one-launch SSP-RK3 step (HYDRO_PARAM_FUSED_RK3): the three stages of a
step as one persistent launch, with per-sub-grid completion counters in place
of the launch boundaries between stages (paper Section VI: the neighbours'
data are read where they lie, with no exchange step between the stages) and,
in mixed precision, the coarse-fine correction run inside the launch.  Its
results equal the three-launch form's bit for bit (same arithmetic in the same
order per cell; only the schedule differs), on the AMR octree and on the full
65536-leaf workload; its waits are bounded and report HYDRO_ERR_TIMEOUT."""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
IN = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))


@pytest.fixture(scope="module")
def hydro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build, hydro as HY
    build.build()
    return HY


def _run(hydro, g, w, U, fused, steps, resync=0, order=0):
    """steps RK3 steps of hydro_rk3_run_cfl from U (host), in the given form;
    returns interiors, dts, totals, speeds and the kernel launches."""
    g.set_param(hydro.PARAM_FUSED_RK3, fused)
    g.set_param(hydro.PARAM_TAU_RESYNC, resync)
    g.set_param(hydro.PARAM_QUEUE_ORDER, order)
    Ud = torch.from_numpy(U).cuda()
    s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
    ids = torch.as_tensor(w.batches.ids, device="cuda")
    ms = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.step(Ud, 0.0, U_out=s1, ids=ids, max_speed=ms)     # first CFL speed
    dts = torch.zeros(steps, dtype=torch.float64, device="cuda")
    tots = torch.zeros((steps, 11), dtype=torch.float64, device="cuda")
    l0 = g.launches
    g.rk3_run_cfl(Ud, 0.4, s1, s2, ms, steps, ids=ids, batch_offsets=w.batches.offsets, dt_out=dts, totals=tots)
    g.sync()
    return (Ud[IN].cpu().numpy(), dts.cpu().numpy(), tots.cpu().numpy(), ms.cpu().numpy()), g.launches - l0


@pytest.mark.parametrize("resync", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cfg", [2, 3])
def test_one_launch_matches_three_launches(hydro, cfg, prec, resync):
    w = W.config(cfg)
    U = w.state()
    if resync:
        rng = np.random.Generator(np.random.PCG64(23))
        U[IN[0], 5:6, IN[2], IN[3], IN[4]] *= rng.uniform(0.5, 1.5, U[IN][:, 5:6].shape)
    g = hydro.HydroGrid(w.grid, precision=prec)
    (a, la), (b, lb) = (_run(hydro, g, w, U, f, 3, resync) for f in (0, 1))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.all(a[1] > 0)
    # per step: the dt kernel, the stage launches (three, and in mixed precision
    # with coarse-fine faces three correction passes; one fused), the totals
    assert lb < la
    if prec == "mixed":   # the batch's own queue order gives the same results
        c, _ = _run(hydro, g, w, U, 1, 3, resync, order=1)
        for x, y in zip(a, c):
            assert np.array_equal(x, y)
    g.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_one_launch_full_size_bit_identical(hydro, prec):
    """The benchmark's workload (65536 sub-grids, 33.5 M cells, 3 levels): one
    step in each form, interiors, dt and totals equal bit for bit."""
    w = W.config(5)
    U = w.state()
    g = hydro.HydroGrid(w.grid, precision=prec)
    a, _ = _run(hydro, g, w, U, 0, 1)
    b, _ = _run(hydro, g, w, U, 1, 1)
    del U
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_one_launch_wait_timeout_is_reported(hydro, prec):
    """Made to wait for inputs that cannot come (one CTA and the queue that
    interleaves the stages of each sub-grid: the CTA's next item is the second
    stage of a sub-grid whose neighbours' first stages are queued behind it),
    the wait runs out after the set number of clock cycles, the launch stops
    taking work and hydro_sync reports HYDRO_ERR_TIMEOUT; the same handle then
    runs a normal step bit-identical to the three-launch form."""
    w = W.config(3)
    U = w.state()
    g = hydro.HydroGrid(w.grid, precision=prec)
    ref, _ = _run(hydro, g, w, U, 0, 1)
    g.set_param(hydro.PARAM_FUSED_RK3, 2)
    g.set_param(hydro.PARAM_STAGE_GRID, 1)
    g.set_param(hydro.PARAM_WAIT_LIMIT, 200000)     # about 0.1 ms
    Ud = torch.from_numpy(U).cuda()
    s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
    g.rk3_step(Ud, 1e-4, s1, s2, ids=torch.as_tensor(w.batches.ids, device="cuda"))
    with pytest.raises(hydro.HydroError) as e:
        g.sync()
    assert e.value.code == -5
    g.sync()                                        # the error word was cleared
    g.set_param(hydro.PARAM_STAGE_GRID, 0)
    g.set_param(hydro.PARAM_WAIT_LIMIT, 2 ** 31 - 1)
    got, _ = _run(hydro, g, w, U, 1, 1)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    g.close()
