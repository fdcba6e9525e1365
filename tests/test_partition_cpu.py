"""Sharded step on CPU ranks: partition + halo exchange against the single domain.

Each gloo rank owns a contiguous Morton range of sub-grids, exchanges the
interiors its neighbours need before every RK stage, and advances its range
with the oracle; the gathered state must equal the single-domain oracle run
bit for bit (ghost values are pure copies and fixed-order means, the stage
reads the same values in the same order)."""
import os
import socket

import numpy as np
import pytest

from paper_2210_06437_gb300 import partition as P
from paper_2210_06437_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

INTERIOR = P.INTERIOR


@pytest.mark.parametrize("cfg,world", [(3, 2), (3, 3), (2, 4)])
def test_plans_are_consistent(cfg, world):
    g = W.config(cfg).grid
    parts = [P.build(g, r, world) for r in range(world)]
    assert sorted(np.concatenate([p.owned for p in parts]).tolist()) == list(range(g.n))
    for p in parts:
        # every neighbour an owned sub-grid reads is local (owned or proxy)
        m = p.n_owned
        nb = p.local.neighbor[:m]
        rel = p.local.neighbor_rel[:m]
        assert np.all(nb[:, :, 0][g.neighbor[p.owned][:, :, 0] >= 0] >= 0)
        assert np.all(nb[rel == 1] >= 0)
        # the local table points at the same sub-grids as the global one
        gids = np.concatenate([p.owned, p.proxies])
        used = g.neighbor[p.owned] >= 0
        assert np.array_equal(gids[nb[used]], g.neighbor[p.owned][used])
        # proxies are exactly the remote neighbours
        assert np.all(p.owner[p.proxies] != p.rank)
        # symmetric send / receive plans
        for q, ids in p.send.items():
            assert np.array_equal(np.sort(ids), np.sort(parts[q].recv[p.rank]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload(cfg):
    """(grid, initial padded state) of a configuration, or of the small AMR blob."""
    if cfg == "blob":
        return H.amr_blob_state()
    w = W.config(cfg)
    return w.grid, w.state()


def _worker(rank, world, port, cfg, steps, out, slabs=False, cw84=0):
    nth = max(1, (os.cpu_count() or 2) // world)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS=str(nth))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        grid, U0 = _workload(cfg)
        p = P.build(grid, rank, world)
        o = oracle.Oracle(p.local, cw84=cw84)
        depth = P.SLAB_CW84 if cw84 & 1 else P.SLAB
        own = np.arange(p.n_owned, dtype=np.int32)
        UL = P.scatter_global(p, U0.copy())
        if slabs:   # proxies start stale: only the exchanged cells may be read
            UL[p.n_owned:][INTERIOR] = np.nan

        def stage(Uin, dt, U0=None, beta=1.0):
            if slabs:
                P.exchange_slabs(p, Uin, dist, depth)
            else:
                P.exchange(p, Uin, dist)
            o.fill_ghosts(Uin)
            Uout = Uin.copy()
            # every sub-grid of the global grid is advanced by this stage (the
            # proxies by their owners), which the flux correction needs to know
            _, ms, st = o.stage(Uin, dt, U0=U0, beta=beta, Uout=Uout, ids=own, nthreads=nth, batch_all=True)
            assert st == 0
            return Uout, P.allreduce_max(ms, dist)

        _, ms = stage(UL, 0.0)
        dts = []
        for _ in range(steps):
            dt = 0.4 / ms[1]
            dts.append(dt)
            U1, ms = stage(UL, dt)
            U2, _ = stage(U1, dt, U0=UL, beta=0.25)
            UL, _ = stage(U2, dt, U0=UL, beta=2.0 / 3.0)
        got = P.gather_owned(p, UL, dist)
        if rank == 0:
            og = oracle.Oracle(grid, cw84=cw84)
            U = og.fill_ghosts(U0.copy())
            _, ms, _ = og.stage(U, 0.0, nthreads=nth)
            for dt in dts:
                assert dt == 0.4 / ms[1]
                U, ms, st = og.rk3_step(U, dt, nthreads=nth)
            out.put(("ok", bool(np.array_equal(got, U[INTERIOR])), float(np.abs(got - U[INTERIOR]).max())))
        dist.barrier()
    except Exception as e:  # report to the parent instead of hanging it
        out.put(("error", rank, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


# the small AMR blob (71 sub-grids, coarse-fine faces between ranks) keeps the
# CPU suite short; the 4096-leaf octree is sharded on the GPU (test_sharded_gpu)
@pytest.mark.parametrize("cfg,world,steps,slabs,cw84", [("blob", 2, 2, False, 0), (1, 2, 3, False, 0),
                                                         ("blob", 2, 2, True, 0), ("blob", 3, 2, True, 0),
                                                         ("blob", 2, 2, True, 3)])
def test_sharded_step_matches_single_domain(oracle_mod, cfg, world, steps, slabs, cw84):
    """slabs: the exchange moves only the cells each receiver reads (face
    slabs; whole interiors of finer proxies); the proxies' other cells then
    hold stale values that no owned sub-grid may read.  cw84: the CW84
    extensions, whose flattening reads four layers (4-layer slabs)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cfg, steps, q, slabs, cw84)) for r in range(world)]
    for pr in procs:
        pr.start()
    msg = q.get(timeout=600)
    for pr in procs:
        pr.join(timeout=120)
    assert msg[0] == "ok", msg
    assert msg[1], "max difference %g" % msg[2]
    assert all(pr.exitcode == 0 for pr in procs)
