"""Slab decomposition of a voxel domain: sub-domains along one axis, one exchange per step.

The method's cost is lattice points times time steps (Sec. 3.4 compares runs on "the same
number of processing units"; Sec. 5 quotes throughput per processor), so a domain too large for
one GPU, or one to be finished sooner, is cut into slabs along its longest axis and each slab is
advanced by its own lbm_domain.  Streaming (Sec. 2.1.1) is the only coupling between cells and
reaches one cell along each axis, so each slab carries a one-cell halo layer on each cut face
(mask value 4 of lbm_create_domain): after every step the 9 post-collision populations that
leave a slab through a cut face are copied into the neighbour's halo layer (lbm_halo_pack on the
sender, lbm_halo_unpack on the receiver), where the neighbour's next step pulls them.  The slabs
then reproduce the undivided domain's fields bit for bit.

  SlabPlan      the split (host logic only): slab ranges, neighbours, the sub-domain geometries
                and the list of transfers of one exchange.
  SlabDomain    every slab on one GPU, exchanging through device buffers on one stream.
  exchange_between_ranks   one slab per process: the same transfers as point-to-point messages
                (torch.distributed isend / irecv: NCCL between GPUs, gloo on the CPU).

The halo exchange needs the A-B streaming scheme (two population arrays): the in-place esoteric
twist writes a cell's outgoing populations into its neighbours' slots, so a cut would split a
cell's writes between two sub-domains.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs as I

HALO = 4  # mask value of a halo cell


@dataclasses.dataclass
class Part:
    index: int
    lo: int              # first interior layer along the split axis (global)
    hi: int              # one past the last interior layer
    low: int | None      # neighbouring part across the low cut face (None: no halo there)
    high: int | None

    @property
    def n_low(self):
        return 0 if self.low is None else 1

    @property
    def n_high(self):
        return 0 if self.high is None else 1


class SlabPlan:
    """Split of a box of shape (nz, ny, nx) into n_parts slabs along `axis` (0 = x, 1 = y, 2 = z;
    default: the longest axis, the highest one on a tie).  A periodic split axis wraps: the first
    and last slabs are neighbours."""

    def __init__(self, shape, periodic=(0, 0, 0), n_parts=2, axis=None):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.ext = (nx, ny, nz)
        if axis is None:
            axis = max(range(3), key=lambda a: (self.ext[a], a))
        self.axis = int(axis)
        self.n_parts = int(n_parts)
        n = self.ext[self.axis]
        if self.n_parts < 1 or n < 2 * self.n_parts:
            raise ValueError(f"cannot cut {n} layers into {n_parts} slabs of at least 2")
        self.periodic = tuple(int(bool(p)) for p in periodic)
        wrap = bool(self.periodic[self.axis]) and self.n_parts > 1
        bounds = [(k * n) // self.n_parts for k in range(self.n_parts + 1)]
        self.parts = []
        for k in range(self.n_parts):
            low = k - 1 if k > 0 else (self.n_parts - 1 if wrap else None)
            high = k + 1 if k < self.n_parts - 1 else (0 if wrap else None)
            self.parts.append(Part(k, bounds[k], bounds[k + 1], low, high))
        # a cut axis is no longer periodic inside a slab: its wrap is an exchange
        sp = list(self.periodic)
        if self.n_parts > 1:
            sp[self.axis] = 0
        self.sub_periodic = tuple(sp)

    # ------------------------------------------------------------------ geometry
    def low_face(self):
        return 2 * self.axis

    def high_face(self):
        return 2 * self.axis + 1

    def layers(self, k):
        """Global layer index along the split axis of every local layer of part k (halo
        layers included, wrapped on a periodic axis)."""
        p = self.parts[k]
        n = self.ext[self.axis]
        return np.array([(i % n) for i in range(p.lo - p.n_low, p.hi + p.n_high)], dtype=np.int64)

    def local_shape(self, k):
        s = list(self.ext)
        s[self.axis] = len(self.layers(k))
        return (s[2], s[1], s[0])

    def interior(self, k):
        """Slice of part k's local layers that it owns (its halo layers excluded)."""
        p = self.parts[k]
        return slice(p.n_low, p.n_low + (p.hi - p.lo))

    def _take(self, arr, k):
        """arr (..., nz, ny, nx) restricted to part k's local layers."""
        return np.take(arr, self.layers(k), axis=arr.ndim - 1 - self.axis)

    def part_geometry(self, g: I.Geometry, k: int) -> I.Geometry:
        """The sub-domain geometry of part k: its layers of the mask (halo layers: 4 where the
        neighbour's cell is fluid, inlet or outlet), the wall links of its own cells with their
        box indices renumbered, the inlet centre in local coordinates, the relaxation-time field
        restricted to its layers, and the split axis no longer periodic."""
        p = self.parts[k]
        mask = self._take(g.mask, k).copy()
        ax = 2 - self.axis  # array axis of the split axis in (nz, ny, nx)
        if p.n_low:
            sl = [slice(None)] * 3
            sl[ax] = 0
            layer = mask[tuple(sl)]
            layer[layer != 0] = HALO
        if p.n_high:
            sl = [slice(None)] * 3
            sl[ax] = mask.shape[ax] - 1
            layer = mask[tuple(sl)]
            layer[layer != 0] = HALO
        links = None
        if g.links is not None and len(g.links[0]):
            cell, beta, q = (np.asarray(a) for a in g.links)
            nz, ny, nx = self.shape
            xyz = np.stack([cell % nx, (cell // nx) % ny, cell // (nx * ny)], axis=1)
            c = xyz[:, self.axis]
            own = (c >= p.lo) & (c < p.hi)
            xyz = xyz[own].copy()
            xyz[:, self.axis] += p.n_low - p.lo
            lz, ly, lx = mask.shape
            links = ((xyz[:, 0] + lx * (xyz[:, 1] + ly * xyz[:, 2])).astype(np.int64),
                     np.asarray(beta)[own].astype(np.uint8), np.asarray(q)[own].astype(np.float64))
        center = list(g.inlet_center)
        center[self.axis] -= p.lo - p.n_low
        tau_cell = None if g.tau_cell is None else self._take(np.asarray(g.tau_cell), k).copy()
        return I.Geometry(mask=mask, periodic=self.sub_periodic, links=links, inlet_center=tuple(center),
                          inlet_radius=g.inlet_radius, tau=g.tau, g0=g.g0, gamp=g.gamp, gomega=g.gomega,
                          wave=g.wave, tau_cell=tau_cell, info=dict(g.info, slab=k, slabs=self.n_parts))

    # ------------------------------------------------------------------ exchange
    def transfers(self, mask=None):
        """One exchange as (source part, source face, destination part, destination face): the
        source packs the populations leaving through its face, the destination unpacks them into
        the halo layer of its face across the same cut.  Listed in the same order on every rank.
        With the global mask, a cut where the layer on either side is solid throughout carries
        nothing (no cell of that layer pulls across it, and the other side has no halo cells)
        and is left out."""
        n = self.ext[self.axis]
        out = []
        for p in self.parts:
            if p.low is not None:
                out.append((p.low, self.high_face(), p.index, self.low_face(), (p.lo - 1) % n, p.lo))
            if p.high is not None:
                out.append((p.high, self.low_face(), p.index, self.high_face(), p.hi % n, p.hi - 1))
        if mask is not None:
            ax = mask.ndim - 1 - self.axis
            live = np.take(mask, np.arange(n), axis=ax).astype(bool).any(axis=tuple(d for d in range(3) if d != ax))
            out = [t for t in out if live[t[4]] and live[t[5]]]
        return [t[:4] for t in out]

    def face_values(self):
        """Values in one exchange buffer: 9 directions x the area of a cut face."""
        a, b = [self.ext[d] for d in range(3) if d != self.axis]
        return 9 * a * b


def exchange_between_ranks(plan: SlabPlan, rank: int, pack, unpack, make_buf, group=None, mask=None):
    """One exchange of the slab held by this rank with its neighbours' ranks (rank k holds part
    k): pack(face, buf) fills a buffer with the populations leaving through a face, unpack(face,
    buf) writes a received buffer into a halo layer, make_buf() gives an empty buffer.  Messages
    carry the destination face as their tag; every rank posts its sends and receives in the
    order of plan.transfers(mask) (mask: the global mask, as every rank has it)."""
    import torch.distributed as dist

    ops, recvs = [], []
    for src, sf, dst, df in plan.transfers(mask):
        if src == rank:
            buf = make_buf()
            pack(sf, buf)
            ops.append(dist.isend(buf, dst, group=group, tag=df))
        if dst == rank:
            buf = make_buf()
            recvs.append((df, buf))
            ops.append(dist.irecv(buf, src, group=group, tag=df))
    for op in ops:
        op.wait()
    for df, buf in recvs:
        unpack(df, buf)


class SlabDomain:
    """Every slab of a split domain on one GPU, advanced in lock step with an exchange after
    each step through device buffers on the slabs' common stream.  Fields and diagnostics are
    reassembled over the slabs' own cells."""

    def __init__(self, g: I.Geometry, n_parts=2, axis=None, storage="fp32", **kw):
        import torch

        from . import lbm

        self.plan = SlabPlan(g.mask.shape, g.periodic, n_parts, axis)
        self.shape = g.mask.shape
        self.transfers = self.plan.transfers(g.mask)
        self.parts = [lbm.Domain.from_geometry(self.plan.part_geometry(g, k), storage=storage, scheme="ab", **kw)
                      for k in range(n_parts)]
        dtype = torch.int32 if storage == "fp32" else torch.int16
        self.bufs = {}
        for src, sf, dst, df in self.transfers:
            n = self.parts[src].halo_size(sf)
            assert n == self.parts[dst].halo_size(df) == self.plan.face_values()
            self.bufs[(src, sf)] = torch.empty(n, dtype=dtype, device=self.parts[src].device)

    def exchange(self):
        tr = self.transfers
        for src, sf, _, _ in tr:
            self.parts[src].halo_pack(sf, self.bufs[(src, sf)])
        for src, sf, dst, df in tr:
            self.parts[dst].halo_unpack(df, self.bufs[(src, sf)])

    def step(self, n=1):
        for _ in range(int(n)):
            for d in self.parts:
                d.step(1)
            self.exchange()

    @property
    def time(self):
        return self.parts[0].time

    def init_equilibrium(self, rho, u):
        """rho (nz, ny, nx), u (3, nz, ny, nx) numpy arrays of the whole box."""
        for k, d in enumerate(self.parts):
            d.init_equilibrium(self.plan._take(rho, k), self.plan._take(u, k))
        self.exchange()

    def macroscopic(self):
        nz, ny, nx = self.shape
        rho = np.zeros((nz, ny, nx), np.float32)
        u = np.zeros((3, nz, ny, nx), np.float32)
        ax = 2 - self.plan.axis
        for k, d in enumerate(self.parts):
            r, uu = d.macroscopic()
            sl = [slice(None)] * 3
            sl[ax] = self.plan.interior(k)
            p = self.plan.parts[k]
            dst = [slice(None)] * 3
            dst[ax] = slice(p.lo, p.hi)
            rho[tuple(dst)] = r[tuple(sl)]
            u[(slice(None),) + tuple(dst)] = uu[(slice(None),) + tuple(sl)]
        return rho, u

    def diagnostics(self):
        ds = [d.diagnostics(raise_unstable=False) for d in self.parts]
        return {"mass": sum(x["mass"] for x in ds), "flux_in": sum(x["flux_in"] for x in ds),
                "flux_out": sum(x["flux_out"] for x in ds), "max_u": max(x["max_u"] for x in ds),
                "n_nonfinite": sum(x["n_nonfinite"] for x in ds), "time": ds[0]["time"]}

    def close(self):
        for d in self.parts:
            d.close()
