"""Partition of an octree grid over ranks, with proxy slots and a halo exchange.

Sub-grids are numbered in Morton order, so each rank owns one contiguous
range of leaves, balanced by leaf count.  A rank's local state holds its owned
sub-grids first and then one proxy slot per remote sub-grid that an owned
sub-grid reads across a face (same-level, coarser or finer neighbour).  Before
every RK stage, ``exchange`` copies the current interiors of those remote
sub-grids into the proxy slots (point-to-point send/recv; the only data-path
communication the sharded step needs); the stage then runs on the local grid
exactly as on a single domain, because it reads neighbours' interiors only.
The maximum signal speed is combined with ``allreduce(MAX)``.

Index logic and data movement only; no solver arithmetic.  The coarse-fine
flux correction of a stage needs a finer neighbour's flux on its face toward
the coarse sub-grid; for a remote finer neighbour that flux is recomputed on
its proxy slot, from the proxy's interior and the ghosts of that face (the
owned coarse sub-grid): the CUDA library takes such proxies as flux-only batch
items (HYDRO_ITEM_FLUX_ONLY, ``flux_only_proxies``), the oracle with
``batch_all``.  ``exchange`` moves whole interiors; ``exchange_slabs`` (and
``exchange_direct`` for partitions held in one process) only what a receiver
reads: 3-layer face slabs of same-level and coarser proxies, whole interiors of
finer ones.  One process per GPU runs the CUDA library on its local grid; CPU
ranks drive the oracle with the same plan, which is how the tests validate it
without several GPUs.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List

import numpy as np

from .workloads import Grid, NF, NG, NP, NX


@dataclasses.dataclass
class Partition:
    rank: int
    world: int
    owned: np.ndarray      # global ids owned by this rank (contiguous Morton range)
    proxies: np.ndarray    # global ids of remote sub-grids held as proxy slots
    local: Grid            # descriptor of owned + proxy slots, local numbering
    owner: np.ndarray      # rank owning each global sub-grid
    send: Dict[int, np.ndarray]  # rank -> global ids this rank sends there each stage
    recv: Dict[int, np.ndarray]  # rank -> global ids received from there (in proxy order)
    glob: Grid = None      # the global grid the plan was cut from

    @property
    def n_owned(self) -> int:
        return len(self.owned)

    def local_index(self, gids: np.ndarray) -> np.ndarray:
        """Local slot of global ids (owned or proxy)."""
        lut = self._lut
        out = lut[np.asarray(gids)]
        assert np.all(out >= 0)
        return out


def ranges(n: int, world: int) -> List[range]:
    """Contiguous, count-balanced ranges of the Morton-ordered leaves."""
    return [range(n * r // world, n * (r + 1) // world) for r in range(world)]


def _needed(grid: Grid, ids: np.ndarray) -> np.ndarray:
    """Global ids read across the faces of the sub-grids ids."""
    nb = grid.neighbor[ids]                       # [m,6,4]
    rel = grid.neighbor_rel[ids]                  # [m,6]
    used = np.zeros_like(nb, dtype=bool)
    used[:, :, 0] = nb[:, :, 0] >= 0
    used[:, :, 1:] = (rel == 1)[:, :, None]
    return np.unique(nb[used])


def build(grid: Grid, rank: int, world: int) -> Partition:
    rs = ranges(grid.n, world)
    owner = np.empty(grid.n, np.int32)
    for r, rg in enumerate(rs):
        owner[rg.start:rg.stop] = r
    owned = np.arange(rs[rank].start, rs[rank].stop, dtype=np.int32)
    need = _needed(grid, owned)
    proxies = need[owner[need] != rank].astype(np.int32)
    gids = np.concatenate([owned, proxies])
    lut = np.full(grid.n, -1, np.int64)
    lut[gids] = np.arange(len(gids))
    m = len(gids)
    nb = np.full((m, 6, 4), -1, np.int32)
    rel = np.zeros((m, 6), np.int8)
    o_nb = grid.neighbor[owned]
    nb[:len(owned)] = np.where(o_nb >= 0, lut[np.maximum(o_nb, 0)], -1)
    rel[:len(owned)] = grid.neighbor_rel[owned]
    # proxy slots are never advanced; a face of a proxy keeps its neighbours
    # where they are all local (the coarse-fine flux correction recomputes a
    # finer proxy's flux on its face toward the owned sub-grid, which needs
    # that face's ghosts); other faces become outflow, which only changes
    # fluxes nobody uses
    for r, gid in enumerate(proxies, start=len(owned)):
        for face in range(6):
            relf = grid.neighbor_rel[gid, face]
            ids = grid.neighbor[gid, face, :4 if relf == 1 else 1]
            if np.all(ids >= 0) and np.all(lut[ids] >= 0):
                nb[r, face, :len(ids)] = lut[ids]
                rel[r, face] = relf
    local = Grid(n=m, dx=grid.dx[gids].copy(), origin=grid.origin[gids].copy(), level=grid.level[gids].copy(),
                 octant=grid.octant[gids].copy(), neighbor=nb, neighbor_rel=rel, periodic=grid.periodic,
                 gamma=grid.gamma, de_switch=grid.de_switch)
    # symmetric plan: rank r sends to rank q the sub-grids q holds as proxies
    send, recv = {}, {}
    for q in range(world):
        if q == rank:
            continue
        qn = _needed(grid, np.arange(rs[q].start, rs[q].stop, dtype=np.int32))
        s = qn[owner[qn] == rank]
        if len(s):
            send[q] = s.astype(np.int32)
        rcv = proxies[owner[proxies] == q]
        if len(rcv):
            recv[q] = rcv
    p = Partition(rank=rank, world=world, owned=owned, proxies=proxies, local=local, owner=owner, send=send,
                  recv=recv, glob=grid)
    p._lut = lut
    return p


INTERIOR = (slice(None), slice(None), slice(NG, NG + NX), slice(NG, NG + NX), slice(NG, NG + NX))


def scatter_global(p: Partition, U_global: np.ndarray) -> np.ndarray:
    """Local state (owned + proxies) cut from a global padded state."""
    return np.ascontiguousarray(U_global[np.concatenate([p.owned, p.proxies])])


def exchange(p: Partition, U_local, dist) -> None:
    """Fill the proxy interiors of U_local (numpy or torch, [m,11,14,14,14])
    with the owners' current interiors.  dist is torch.distributed."""
    import torch
    is_np = isinstance(U_local, np.ndarray)
    T = torch.from_numpy(U_local) if is_np else U_local
    reqs, bufs = [], []
    for q, gids in sorted(p.send.items()):
        li = torch.as_tensor(p.local_index(gids), device=T.device)
        buf = T[li][:, :, NG:NG + NX, NG:NG + NX, NG:NG + NX].contiguous()
        bufs.append(buf)
        reqs.append(dist.isend(buf, dst=q))
    recvs = []
    for q, gids in sorted(p.recv.items()):
        buf = torch.empty((len(gids), NF, NX, NX, NX), dtype=T.dtype, device=T.device)
        recvs.append((gids, buf))
        reqs.append(dist.irecv(buf, src=q))
    for r in reqs:
        r.wait()
    for gids, buf in recvs:
        li = torch.as_tensor(p.local_index(gids), device=T.device)
        T[li, :, NG:NG + NX, NG:NG + NX, NG:NG + NX] = buf


# ---------------------------------------------------------------------------
# slab exchange: only the cells a receiver reads
# ---------------------------------------------------------------------------

SLAB = 3          # layers of a proxy that a same-level or finer owned neighbour reads across a face
SLAB_CW84 = 4     # with the CW84 flattening, whose pressures reach one layer further
WHOLE = -1        # a finer proxy: the whole interior (the coarse owner reads six fine layers for its
                  # 2x2x2 halo means, and the proxy's boundary flux is recomputed from it)


def slab_entries(grid: Grid, gids: np.ndarray, owner: np.ndarray, reader: int) -> list:
    """(gid, face) pieces of the proxies gids that rank `reader` reads: face
    slabs (of `depth` layers, see _region) where a reader's sub-grid is a same-level or finer
    neighbour across that face, the whole interior (face WHOLE) where a
    reader's sub-grid is coarser.  Both sides of an exchange derive the same
    list from the global grid."""
    out = []
    for g in np.asarray(gids).tolist():
        whole, faces = False, []
        for face in range(6):
            relf = int(grid.neighbor_rel[g, face])
            nbs = grid.neighbor[g, face, :4 if relf == 1 else 1]
            if not np.any((nbs >= 0) & (owner[np.maximum(nbs, 0)] == reader)):
                continue
            if relf == -1:
                whole = True
            else:
                faces.append(face)
        out.extend([(g, WHOLE)] if whole else [(g, f) for f in faces])
    return out


def _region(face: int, depth: int = SLAB):
    """Index of the padded interior cells of a piece (a face slab of `depth`
    layers, or WHOLE) within [f, k, j, i].  A same-level reader's halo reads
    three layers (four with the CW84 flattening); a finer reader's, by
    injection, at most two coarse layers."""
    I = slice(NG, NG + NX)
    if face == WHOLE:
        return (slice(None), I, I, I)
    a, side = face // 2, face % 2
    cut = slice(NG, NG + depth) if side == 0 else slice(NG + NX - depth, NG + NX)
    sl = [slice(None), I, I, I]
    sl[3 - a] = cut
    return tuple(sl)


def pack_pieces(U, entries, local_index, depth: int = SLAB) -> "object":
    """The cells of `entries` from the local state U (torch, [m,11,14,14,14]) as one flat tensor."""
    import torch
    if not entries:
        return torch.empty(0, dtype=U.dtype, device=U.device)
    li = local_index(np.array([g for g, _ in entries]))
    return torch.cat([U[int(l)][_region(f, depth)].reshape(-1) for l, (_, f) in zip(li, entries)])


def unpack_pieces(U, entries, local_index, buf, depth: int = SLAB) -> None:
    """Write the flat buffer of pack_pieces into the proxy slots of U."""
    if not entries:
        return
    li = local_index(np.array([g for g, _ in entries]))
    o = 0
    for l, (_, f) in zip(li, entries):
        view = U[int(l)][_region(f, depth)]
        n = view.numel()
        view.copy_(buf[o:o + n].view(view.shape))
        o += n


def exchange_slabs(p: Partition, U_local, dist, depth: int = SLAB) -> int:
    """exchange() with only the cells each receiver reads (face slabs of
    `depth` layers, whole interiors of finer proxies); returns the bytes this
    rank sent."""
    import torch
    is_np = isinstance(U_local, np.ndarray)
    T = torch.from_numpy(U_local) if is_np else U_local
    reqs, keep, sent = [], [], 0
    for q, gids in sorted(p.send.items()):
        buf = pack_pieces(T, slab_entries(p.glob, gids, p.owner, q), p.local_index, depth)
        keep.append(buf)
        sent += buf.numel() * buf.element_size()
        reqs.append(dist.isend(buf, dst=q))
    recvs = []
    for q, gids in sorted(p.recv.items()):
        entries = slab_entries(p.glob, gids, p.owner, p.rank)
        n = sum(T[0][_region(f, depth)].numel() for _, f in entries)
        buf = torch.empty(n, dtype=T.dtype, device=T.device)
        recvs.append((entries, buf))
        reqs.append(dist.irecv(buf, src=q))
    for r in reqs:
        r.wait()
    for entries, buf in recvs:
        unpack_pieces(T, entries, p.local_index, buf, depth)
    return sent


def exchange_direct(parts: List[Partition], states: list, depth: int = SLAB) -> int:
    """The slab exchange between partitions held in one process (device
    copies): every rank's proxies receive, from their owners' local states,
    the cells it reads (face slabs of `depth` layers).  Returns the bytes moved."""
    moved = 0
    for r, p in enumerate(parts):
        for q, gids in sorted(p.recv.items()):
            entries = slab_entries(p.glob, gids, p.owner, r)
            buf = pack_pieces(states[q], entries, parts[q].local_index, depth)
            moved += buf.numel() * buf.element_size()
            unpack_pieces(states[r], entries, p.local_index, buf, depth)
    return moved


def flux_only_proxies(p: Partition) -> np.ndarray:
    """Local slots of the finer proxies next to an owned coarse sub-grid: a
    stage lists them as flux-only items (their boundary fluxes feed the owned
    sub-grid's coarse-fine correction; their owners advance them)."""
    m = p.n_owned
    nb = p.local.neighbor[:m]
    rel = p.local.neighbor_rel[:m]
    ids = nb[rel == 1].reshape(-1)
    return np.unique(ids[ids >= m]).astype(np.int32)


def allreduce_max(x: np.ndarray, dist) -> np.ndarray:
    import torch
    t = torch.as_tensor(np.asarray(x, np.float64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.numpy()


def gather_owned(p: Partition, U_local: np.ndarray, dist, root: int = 0):
    """Owned interiors of every rank assembled on root as a global array
    (other ranks return None)."""
    import torch
    mine = torch.from_numpy(np.ascontiguousarray(U_local[:p.n_owned][INTERIOR]))
    if p.rank != root:
        dist.send(mine, dst=root)
        return None
    out = [None] * p.world
    out[root] = mine
    for q in range(p.world):
        if q == root:
            continue
        n_q = len(ranges(len(p.owner), p.world)[q])
        buf = torch.empty((n_q, NF, NX, NX, NX), dtype=torch.float64)
        dist.recv(buf, src=q)
        out[q] = buf
    return torch.cat(out).numpy()
