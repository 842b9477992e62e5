"""One mesh split over several processes (the parallel transport of Sec. 2.4):
host-side logic of the slab partition.

The mesh of n0 x n1 x n2 cells (cell index i + n0 (j + n1 k)) is cut into
`world` slabs of whole cell layers along k.  Rank r owns layers
[k_lo, k_hi) and holds a sub-mesh of layers [g_lo, g_hi) = [k_lo - h, k_hi + h)
clipped to the mesh (h halo layers), with those layers' vertices and Q2
nodes.  A cell keeps its global order in the sub-mesh: local index = global
index - shift, shift = n0 n1 g_lo, so the lowest-index rule decides shared
faces the same way.

Every rank advances the particles of its own cells on its sub-mesh; their
stage points and new positions may fall in halo cells, whose data it holds.
After the step the store is sorted by (cell, id): the particles that moved
into halo layers below k_lo are its first cell_off[own_lo] slots, those that
moved above k_hi its slots from cell_off[own_hi] on.  Those two ranges go to
the neighbours with their cells in global numbering, so that the receiver
does not search (Sec. 2.4); each rank keeps its own cells' particles, adds
the received ones and re-sorts (pic_merge_particles).  Two halo layers hold
every stage point of a particle that moves at most one cell per step (CFL
<= 1); a point beyond them is outside the sub-mesh and counts as lost.

The exchange is one round of point-to-point messages with the two
neighbours (counts, then the payload), over torch.distributed: NCCL between
GPUs, gloo in the CPU tests of the protocol.  There is no other collective on
the data path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Slab:
    n: tuple          # global cells per axis (n0, n1, n2)
    rank: int
    world: int
    k_lo: int         # owned layers [k_lo, k_hi)
    k_hi: int
    g_lo: int         # held layers [g_lo, g_hi) (owned plus halo)
    g_hi: int

    @property
    def layer(self) -> int:
        return self.n[0] * self.n[1]

    @property
    def local_n(self) -> tuple:
        return (self.n[0], self.n[1], self.g_hi - self.g_lo)

    @property
    def shift(self) -> int:
        """global cell index - local cell index"""
        return self.layer * self.g_lo

    @property
    def own_lo(self) -> int:
        """first owned cell, local numbering"""
        return self.layer * (self.k_lo - self.g_lo)

    @property
    def own_hi(self) -> int:
        return self.layer * (self.k_hi - self.g_lo)

    @property
    def owned_cells(self) -> int:
        return self.layer * (self.k_hi - self.k_lo)


def slab_bounds(n2: int, world: int) -> list[tuple[int, int]]:
    """Owned layers of each rank: contiguous, as even as whole layers allow."""
    if world < 1 or n2 < world:
        raise ValueError("need 1 <= world <= %d layers (got %d)" % (n2, world))
    return [(r * n2 // world, (r + 1) * n2 // world) for r in range(world)]


def make_slab(n, rank: int, world: int, halo: int = 2) -> Slab:
    n = tuple(int(v) for v in n)
    if len(n) != 3:
        raise ValueError("slab partition needs a 3D mesh")
    k_lo, k_hi = slab_bounds(n[2], world)[rank]
    return Slab(n, rank, world, k_lo, k_hi, max(0, k_lo - halo), min(n[2], k_hi + halo))


def slice_vertices(X: np.ndarray, s: Slab) -> np.ndarray:
    """Vertices [3][nv] of the held layers (vertex layers g_lo .. g_hi)."""
    nv0, nv1 = s.n[0] + 1, s.n[1] + 1
    Xg = X.reshape(3, s.n[2] + 1, nv1, nv0)
    return np.ascontiguousarray(Xg[:, s.g_lo: s.g_hi + 1].reshape(3, -1))


def slice_nodes(U: np.ndarray, s: Slab) -> np.ndarray:
    """Q2 nodal values [3][nq] of the held layers (node layers 2 g_lo .. 2 g_hi)."""
    nq0, nq1 = 2 * s.n[0] + 1, 2 * s.n[1] + 1
    Ug = U.reshape(U.shape[0], 2 * s.n[2] + 1, nq1, nq0)
    return np.ascontiguousarray(Ug[:, 2 * s.g_lo: 2 * s.g_hi + 1].reshape(U.shape[0], -1))


def owned_per_cell(s: Slab, ppc: int) -> np.ndarray:
    """Particles per local cell for a uniform seeding of the owned cells."""
    per = np.zeros(s.layer * (s.g_hi - s.g_lo), dtype=np.uint32)
    per[s.own_lo: s.own_hi] = ppc
    return per


def first_id(s: Slab, ppc: int) -> int:
    """Global id of the rank's first particle under a uniform seeding of the
    whole mesh (ids follow cells)."""
    return s.layer * s.k_lo * ppc


def leaving_ranges(cell_off_lo: int, cell_off_hi: int, n: int) -> tuple[tuple[int, int], tuple[int, int]]:
    """(first, count) of the particles below and above the owned layers in a
    store sorted by cell: [0, off[own_lo]) and [off[own_hi], n)."""
    return (0, cell_off_lo), (cell_off_hi, n - cell_off_hi)


PAYLOAD = ("x", "xhat", "id", "cell", "props")


def _empty_payload(template: dict, n: int, device) -> dict:
    import torch

    return {k: torch.empty((template[k].shape[0], n) if template[k].dim() == 2 else (n,), dtype=template[k].dtype,
                           device=device) for k in PAYLOAD}


def swap_with_neighbours(send_down: dict | None, send_up: dict | None, rank: int, world: int, device, group=None):
    """One exchange round: send_down to rank - 1, send_up to rank + 1; returns
    what rank - 1 and rank + 1 sent (None where there is no neighbour).  Per
    pair the counts go first (one int64 each way), then each payload tensor,
    the lower rank sending first.  Odd ranks serve their upper neighbour
    first and even ranks their lower one, so that blocking transports (gloo)
    pair up without deadlock along the chain."""
    import torch
    import torch.distributed as dist

    partners = []
    if rank > 0:
        partners.append((rank - 1, send_down, "down"))
    if rank + 1 < world:
        partners.append((rank + 1, send_up, "up"))
    if rank % 2 == 1:
        partners.reverse()
    got = {}
    for peer, out, tag in partners:
        c_out = torch.tensor([int(out["id"].shape[0])], dtype=torch.int64, device=device)
        c_in = torch.zeros(1, dtype=torch.int64, device=device)
        first = rank < peer
        if first:
            dist.send(c_out, peer, group=group)
            dist.recv(c_in, peer, group=group)
        else:
            dist.recv(c_in, peer, group=group)
            dist.send(c_out, peer, group=group)
        inc = _empty_payload(out, int(c_in.item()), device)
        for k in PAYLOAD:
            ops = [("s", out[k]), ("r", inc[k])] if first else [("r", inc[k]), ("s", out[k])]
            for kind, t in ops:
                if t.numel() == 0:
                    continue
                if kind == "s":
                    dist.send(t.contiguous(), peer, group=group)
                else:
                    dist.recv(t, peer, group=group)
        got[tag] = inc
    return got.get("down"), got.get("up")


def concat(parts: list) -> dict | None:
    import torch

    parts = [p for p in parts if p is not None and p["id"].shape[0] > 0]
    if not parts:
        return None
    return {k: torch.cat([p[k] for p in parts], dim=-1) for k in PAYLOAD}


def export_leaving(store, s: Slab):
    """The particles of a store sorted by cell that lie below and above the
    owned layers, with their cells in global numbering: (down, up)."""
    off = store.cell_offsets()
    lo, hi, n = (int(v) for v in off[[s.own_lo, s.own_hi, off.shape[0] - 1]].tolist())
    (f0, c0), (f1, c1) = leaving_ranges(lo, hi, n)
    return store.export_range(f0, c0, cell_shift=s.shift), store.export_range(f1, c1, cell_shift=s.shift)


def merge_incoming(store, s: Slab, from_below: dict | None, from_above: dict | None):
    """Keep the owned cells' particles, add the received ones (cells in
    global numbering), re-sort."""
    store.merge(s.own_lo, s.own_hi, concat([from_below, from_above]), cell_shift=-s.shift)


def exchange_step(store, s: Slab, device, group=None):
    """After a time step of `store`: hand the particles that left the owned
    layers to the neighbours and merge what they send.  Returns the numbers
    sent down and up."""
    down, up = export_leaving(store, s)
    from_below, from_above = swap_with_neighbours(down, up, s.rank, s.world, device, group)
    merge_incoming(store, s, from_below, from_above)
    return int(down["id"].shape[0]), int(up["id"].shape[0])
