"""Checkpoint and resume of a multi-step run.

A run of K + M SSP-RK3 steps with the device-chosen (lagged CFL) time step
and per-step totals is compared with a run of K steps that is saved to a file
(the packed interiors, the lagged maximum signal speed that sets the next dt,
the step counter and the dt history), torn down, restored into a new handle
and new device buffers, and continued for M steps: the two end states, dt
sequences and totals are identical bit for bit, in both precisions.
"""
import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, M = 2, 2


@pytest.fixture(scope="module")
def hydro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build, hydro as HY
    build.build()
    return HY


def _start(hydro, w, prec, U_host):
    g = hydro.HydroGrid(w.grid, precision=prec)
    U = torch.from_numpy(U_host).cuda()
    s1, s2 = torch.empty_like(U), torch.empty_like(U)
    ids = torch.as_tensor(w.batches.ids, device="cuda")
    return g, U, s1, s2, ids


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_checkpoint_resume_is_bit_exact(hydro, prec, tmp_path):
    w = W.config(3)
    U0 = w.state()
    offs = w.batches.offsets
    # uninterrupted: K + M steps
    g, U, s1, s2, ids = _start(hydro, w, prec, U0)
    ms = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.step(U, 0.0, U_out=s1, ids=ids, batch_offsets=offs, max_speed=ms)      # first CFL speed
    dts = torch.zeros(K + M, dtype=torch.float64, device="cuda")
    tots = torch.zeros((K + M, 11), dtype=torch.float64, device="cuda")
    g.rk3_run_cfl(U, 0.4, s1, s2, ms, K + M, ids=ids, batch_offsets=offs, dt_out=dts, totals=tots)
    g.sync()
    ref = (g.pack(U).cpu().numpy(), dts.cpu().numpy(), tots.cpu().numpy())
    g.close()
    del U, s1, s2
    # K steps, save, tear down
    g, U, s1, s2, ids = _start(hydro, w, prec, U0)
    ms = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.step(U, 0.0, U_out=s1, ids=ids, batch_offsets=offs, max_speed=ms)
    dts = torch.zeros(K, dtype=torch.float64, device="cuda")
    tots = torch.zeros((K, 11), dtype=torch.float64, device="cuda")
    g.rk3_run_cfl(U, 0.4, s1, s2, ms, K, ids=ids, batch_offsets=offs, dt_out=dts, totals=tots)
    g.sync()
    path = tmp_path / "checkpoint.npz"
    np.savez(path, interiors=g.pack(U).cpu().numpy(), max_speed=ms.cpu().numpy(), step=K, dts=dts.cpu().numpy(),
             totals=tots.cpu().numpy())
    g.close()
    del U, s1, s2, ms
    torch.cuda.empty_cache()
    # restore into a new handle and new buffers (ghost cells are never read)
    ck = np.load(path)
    assert int(ck["step"]) == K
    g = hydro.HydroGrid(w.grid, precision=prec)
    U = torch.full(U0.shape, float("nan"), dtype=torch.float64, device="cuda")
    g.unpack(torch.from_numpy(ck["interiors"]).cuda(), U)
    s1, s2 = torch.empty_like(U), torch.empty_like(U)
    ids = torch.as_tensor(w.batches.ids, device="cuda")
    ms = torch.from_numpy(ck["max_speed"]).cuda()
    dts = torch.zeros(M, dtype=torch.float64, device="cuda")
    tots = torch.zeros((M, 11), dtype=torch.float64, device="cuda")
    g.rk3_run_cfl(U, 0.4, s1, s2, ms, M, ids=ids, batch_offsets=offs, dt_out=dts, totals=tots)
    g.sync()
    got = (g.pack(U).cpu().numpy(), np.concatenate([ck["dts"], dts.cpu().numpy()]),
           np.concatenate([ck["totals"], tots.cpu().numpy()]))
    g.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
