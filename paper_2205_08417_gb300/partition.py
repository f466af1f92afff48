"""A step split over ranks: Morton-range cell partitions with halo layers and their exchange.

The paper runs its solvers with the cells split over shared-memory workers that synchronise
between the phases of a step (Sec. 6, "Parallel Scaling"). Here each rank owns a contiguous range
of the mesh's cells (the meshes are Morton-ordered, so a range is a compact region) and steps a
local mesh made of its own triangles plus `layers` layers of its neighbours' triangles (the
halo). Before each step the halo rows of u, and of alpha (the closure's warm start), are
refreshed from their owners; the rank then runs the unchanged single-GPU step on its local mesh
and keeps the results of its own cells. How many layers make the owned cells' results exact:
  - first order: 1 (the flux of a cell reads the ansatz of its face neighbours, which their own
    u determines);
  - second order with Heun (order 2): 4 (a stage's face values need the neighbours' gradients,
    which need the neighbours' neighbours, and the second stage repeats that on the first
    stage's result).
Exchanging alpha as well keeps every halo closure on its owner's Newton start: the outer halo
cells' second-stage inputs are not exact, and a Newton iterate depends on its start at the
rounding level, so without it the owned cells would match the single-rank step only to the
closure tolerance.
The discrete adjoint runs the transposed map: a rank applies the transposed step to its owned
cells' adjoint rows (zero on its halo), which leaves contributions on its halo rows that belong to
the owners of those cells; reverse_exchange sends them back and adds them there (the transpose of
the forward exchange: a gather becomes a scatter-add).
This module holds only the host-side bookkeeping (partition, local mesh, send and receive lists)
and the exchanges' sequencing; the rows are packed and unpacked by callables the caller passes
(kitrt.gather_rows / kitrt.scatter_rows / kitrt.scatter_add_rows for device arrays) and moved with
torch.distributed point-to-point operations (NCCL between GPUs; gloo between CPU processes in the
tests).
"""
from __future__ import annotations

import numpy as np


def cell_ranges(C: int, nranks: int):
    """Contiguous owned ranges [lo, hi) of a C-cell mesh over nranks ranks."""
    return [(C * r // nranks, C * (r + 1) // nranks) for r in range(nranks)]


def halo_cells(nbr: np.ndarray, lo: int, hi: int, layers: int) -> np.ndarray:
    """Global indices of the cells within `layers` face-neighbour steps of [lo, hi), outside it,
    ordered by layer and then by index."""
    C = nbr.shape[0]
    inside = np.zeros(C, dtype=bool)
    inside[lo:hi] = True
    frontier = np.arange(lo, hi)
    out = []
    for _ in range(layers):
        nb = nbr[frontier].ravel()
        nb = np.unique(nb[nb >= 0])
        new = nb[~inside[nb]]
        inside[new] = True
        out.append(new)
        frontier = new
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


class Partition:
    """Rank `rank`'s share of a mesh (vertices xy [V, 2], triangles tri [C, 3], face neighbours
    nbr [C, 3] with -1 on the boundary) split over `nranks` ranks."""

    def __init__(self, xy: np.ndarray, tri: np.ndarray, nbr: np.ndarray, rank: int, nranks: int,
                 layers: int = 1):
        if not 0 <= rank < nranks or layers < 0:
            raise ValueError("bad rank or layer count")
        C = tri.shape[0]
        self.rank, self.nranks, self.layers = rank, nranks, layers
        ranges = cell_ranges(C, nranks)
        self.lo, self.hi = ranges[rank]
        owner = np.empty(C, dtype=np.int64)
        for r, (a, b) in enumerate(ranges):
            owner[a:b] = r
        halos = [halo_cells(nbr, a, b, layers) for a, b in ranges]
        # local cells: own range first (in order), then the halo
        self.cells = np.concatenate([np.arange(self.lo, self.hi), halos[rank]]).astype(np.int64)
        self.n_owned = self.hi - self.lo
        g2l = np.full(C, -1, dtype=np.int64)
        g2l[self.cells] = np.arange(self.cells.size)
        # receive from r: my halo cells that r owns; send to r: my cells in r's halo (both sides
        # list the cells in increasing global index)
        self.recv, self.send = {}, {}
        mine = halos[rank]
        for r in range(nranks):
            if r == rank:
                continue
            got = np.sort(mine[owner[mine] == r])
            give = np.sort(halos[r][owner[halos[r]] == rank])
            if got.size:
                self.recv[r] = g2l[got].astype(np.int32)
            if give.size:
                self.send[r] = g2l[give].astype(np.int32)
        # local mesh: the local cells' triangles, each with its vertex order, the vertices renumbered
        # in increasing order
        ltri = tri[self.cells]
        verts, inv = np.unique(ltri.ravel(), return_inverse=True)
        self.xy = np.ascontiguousarray(xy[verts], dtype=np.float64)
        self.tri = np.ascontiguousarray(inv.reshape(-1, 3), dtype=np.int32)

    def local(self, global_rows: np.ndarray) -> np.ndarray:
        """Rows of a global per-cell array for the local cells."""
        return np.ascontiguousarray(global_rows[self.cells])

    def exchange(self, u, pack, unpack, empty, dist):
        """Refresh the halo rows of a local per-cell array u (the state, the closure's alpha)
        from their owners. pack(u, idx) returns the
        rows idx of u as a contiguous buffer, unpack(buf, idx, u) writes them back, empty(k)
        makes a receive buffer of k rows; dist is torch.distributed (initialised). All ranks call
        it together; sends and receives are posted at once and waited for."""
        reqs, inbox, outbox = [], {}, []
        for r, idx in sorted(self.send.items()):
            outbox.append(pack(u, idx))  # kept alive until the sends complete
            reqs.append(dist.isend(outbox[-1], r))
        for r, idx in sorted(self.recv.items()):
            inbox[r] = empty(idx.size)
            reqs.append(dist.irecv(inbox[r], r))
        for q in reqs:
            q.wait()
        for r, idx in sorted(self.recv.items()):
            unpack(inbox[r], idx, u)

    def reverse_exchange(self, v, pack, unpack_add, empty, dist):
        """Transpose of exchange(): send the halo rows of a local per-cell array v (contributions of
        this rank's owned rows to cells other ranks own) to their owners, and add the rows received
        for this rank's cells into v. pack(v, idx) returns rows idx of v as a contiguous buffer,
        unpack_add(buf, idx, v) adds buffer row k to row idx[k] of v, empty(k) makes a receive
        buffer. All ranks call it together; the received rows are added in increasing rank order.
        The halo rows of v are left as they were (the caller zeroes them if it reuses v)."""
        reqs, inbox, outbox = [], {}, []
        for r, idx in sorted(self.recv.items()):
            outbox.append(pack(v, idx))
            reqs.append(dist.isend(outbox[-1], r))
        for r, idx in sorted(self.send.items()):
            inbox[r] = empty(idx.size)
            reqs.append(dist.irecv(inbox[r], r))
        for q in reqs:
            q.wait()
        for r, idx in sorted(self.send.items()):
            unpack_add(inbox[r], idx, v)
