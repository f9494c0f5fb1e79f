"""Host logic of the slab decomposition (paper_2101_11107_gb300/slabs.py), on the CPU:

  * the plan partitions the split axis, every halo layer holds the neighbour's layer next to the
    cut (4 where that cell is fluid), the slabs' own layers reassemble the mask, the wall links
    and the relaxation-time field, and inlet centres move to local coordinates;
  * one exchange between two and three gloo ranks (one slab per rank) delivers every buffer to
    the right rank and halo face: each rank packs values that name their origin (rank, face,
    direction, position) and checks what it unpacks against the plan.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2101_11107_gb300 import inputs as I
from paper_2101_11107_gb300 import slabs as S

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _layer(a, axis, i):
    return np.take(a, i, axis=a.ndim - 1 - axis)


@pytest.mark.parametrize("case,n_parts", [("pipe", 2), ("pipe", 3), ("aneurysm", 2), ("aneurysm", 3),
                                          ("ragged", 4)])
def test_plan_geometry(case, n_parts):
    if case == "pipe":  # periodic along the split axis (z): the first and last slabs meet
        g = I.pipe(16, 16, 40, 6.0, tau=0.6, g0=(0, 0, 1e-5), bouzidi=True)
    elif case == "aneurysm":
        g = I.aneurysm(3, edge=48, period=200.0, reynolds=30.0)
    else:
        g = I.inlet_pipe(45, 11, 13, 4.4, u_peak=0.02, tau=0.7, bouzidi=True)
    plan = S.SlabPlan(g.mask.shape, g.periodic, n_parts)
    ax = plan.axis
    n = plan.ext[ax]
    assert plan.ext[ax] == max(plan.ext)
    own = np.concatenate([np.arange(p.lo, p.hi) for p in plan.parts])
    assert np.array_equal(own, np.arange(n))
    wrap = bool(g.periodic[ax])
    assert plan.sub_periodic[ax] == 0 and all(plan.sub_periodic[d] == g.periodic[d] for d in range(3) if d != ax)
    n_links = 0
    for k, p in enumerate(plan.parts):
        sub = plan.part_geometry(g, k)
        m = sub.mask
        assert m.shape == plan.local_shape(k)
        # own layers are the global mask's layers, untouched
        own_layers = _layer(m, ax, np.arange(plan.interior(k).start, plan.interior(k).stop))
        assert np.array_equal(own_layers, _layer(g.mask, ax, np.arange(p.lo, p.hi)))
        assert not np.any(own_layers == S.HALO)
        # halo layers: the neighbour's layer next to the cut, 4 where fluid
        if p.low is not None:
            src = _layer(g.mask, ax, (p.lo - 1) % n)
            assert np.array_equal(_layer(m, ax, 0), np.where(src != 0, S.HALO, 0))
            assert (p.lo - 1) % n == plan.parts[p.low].hi - 1
        else:
            assert p.lo == 0 and not wrap
        if p.high is not None:
            src = _layer(g.mask, ax, p.hi % n)
            assert np.array_equal(_layer(m, ax, m.shape[2 - ax] - 1), np.where(src != 0, S.HALO, 0))
            assert p.hi % n == plan.parts[p.high].lo
        # links: only the slab's own cells, renumbered to the same cells
        if sub.links is not None:
            lz, ly, lx = m.shape
            c = sub.links[0]
            xyz = np.stack([c % lx, (c // lx) % ly, c // (lx * ly)], axis=1)
            assert np.all(m.reshape(-1)[c] == 1)
            xyz[:, ax] += p.lo - p.n_low
            nz, ny, nx = g.mask.shape
            gi = xyz[:, 0] + nx * (xyz[:, 1] + ny * xyz[:, 2])
            gl = {(int(a), int(b)): float(q) for a, b, q in zip(*g.links)}
            for a, b, q in zip(gi, sub.links[1], sub.links[2]):
                assert gl[(int(a), int(b))] == q
            n_links += len(c)
        if g.tau_cell is not None:
            assert np.array_equal(_layer(sub.tau_cell, ax, np.arange(plan.interior(k).start, plan.interior(k).stop)),
                                  _layer(g.tau_cell, ax, np.arange(p.lo, p.hi)))
        assert sub.inlet_center[ax] == g.inlet_center[ax] - (p.lo - p.n_low)
    assert n_links == (0 if g.links is None else len(g.links[0]))
    # every transfer pairs a slab's face with the neighbour's opposite face across one cut
    for src, sf, dst, df in plan.transfers():
        assert {sf, df} == {2 * ax, 2 * ax + 1} and sf != df
        assert (plan.parts[dst].low == src) if df == 2 * ax else (plan.parts[dst].high == src)


def test_plan_rejects_too_many_parts():
    with pytest.raises(ValueError):
        S.SlabPlan((8, 8, 8), (0, 0, 0), 5)
    p = S.SlabPlan((8, 8, 8), (0, 0, 1), 1)
    assert p.transfers() == [] and p.sub_periodic == (0, 0, 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _code(rank, face, j, p):
    return rank * 1_000_000 + face * 100_000 + j * 10_000 + p


def _rank(rank, world, port, shape, periodic, out):
    sys.path.insert(0, ROOT)
    from paper_2101_11107_gb300 import slabs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = slabs.SlabPlan(shape, periodic, world)
        nv = plan.face_values()
        area = nv // 9
        got = {}

        def pack(face, buf):
            j, p = np.divmod(np.arange(nv), area)
            buf.copy_(torch.from_numpy(_code(rank, face, j, p).astype(np.int64)))

        def unpack(face, buf):
            got[face] = buf.numpy().copy()

        slabs.exchange_between_ranks(plan, rank, pack, unpack, lambda: torch.empty(nv, dtype=torch.int64))
        out[rank] = {f: v.tolist() for f, v in got.items()}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,periodic", [(2, (40, 8, 12), (0, 0, 1)), (2, (12, 8, 40), (0, 0, 0)),
                                                  (3, (30, 8, 8), (1, 1, 1))])
def test_exchange_between_gloo_ranks(world, shape, periodic):
    """Each rank unpacks, on every halo face, exactly the buffer its neighbour across that cut
    packed on its opposite face: two ranks on a wrapped axis (both cuts between the same pair),
    two ranks on an open axis (one cut), three ranks on a wrapped axis."""
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(world, port, shape, periodic, out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    plan = S.SlabPlan(shape, periodic, world)
    area = plan.face_values() // 9
    j, p = np.divmod(np.arange(9 * area), area)
    n_recv = 0
    for src, sf, dst, df in plan.transfers():
        assert np.array_equal(np.array(res[dst][df]), _code(src, sf, j, p)), (src, sf, dst, df)
        n_recv += 1
    assert n_recv == sum(len(v) for v in res.values())
    assert n_recv == (2 * world if periodic[plan.axis] else 2 * (world - 1))


def test_cut_through_solid_layers_carries_nothing():
    """A cut with a layer that is solid throughout on one side drops both of its transfers: the
    other side has no halo cells there, and no cell of the solid layer pulls across."""
    mask = np.zeros((24, 8, 8), np.uint8)
    mask[0:10, 2:6, 2:6] = 1   # fluid in z = 0..9 only: the cut at z = 12 meets solid layers
    plan = S.SlabPlan(mask.shape, (0, 0, 0), 2)
    assert plan.transfers() != [] and plan.transfers(mask) == []
    g = I.Geometry(mask=mask)
    assert not np.any(plan.part_geometry(g, 1).mask == S.HALO)
    mask[11:13, 2:6, 2:6] = 1  # both layers at the cut (z = 11, 12) now hold fluid
    assert len(plan.transfers(mask)) == 2
