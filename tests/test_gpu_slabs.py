"""Slab decomposition on one GPU: the sub-domains of a split domain, each its own lbm_domain,
exchanging the face-crossing populations through device buffers after every step
(lbm_halo_pack / lbm_halo_unpack), against the undivided domain (A-B scheme, same launch
configuration).  Every cell is updated by the same arithmetic on the same values, so the fields
must agree bit for bit; the diagnostics, summed over the slabs in another order, to 1e-12.
"""
import numpy as np
import pytest

from paper_2101_11107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402
from paper_2101_11107_gb300 import slabs as S  # noqa: E402


def _compare(g, n_parts, steps, storage="fp32", init=None, axis=None):
    whole = lbm.Domain.from_geometry(g, storage=storage, scheme="ab")
    split = S.SlabDomain(g, n_parts, axis=axis, storage=storage)
    assert sum(d.info()["n_fluid"] for d in split.parts) == whole.info()["n_fluid"] == g.nfluid
    # a slab whose cuts meet solid layers on the far side has no halo cells there
    assert sum(d.info()["n_halo"] for d in split.parts) > 0
    if init is not None:
        whole.init_equilibrium(*init)
        split.init_equilibrium(*init)
    for chunk in (steps // 3, steps - steps // 3):
        whole.step(chunk)
        split.step(chunk)
        r0, u0 = whole.macroscopic()
        r1, u1 = split.macroscopic()
        assert np.array_equal(r0, r1) and np.array_equal(u0, u1)
    d0, d1 = whole.diagnostics(), split.diagnostics()
    for key in ("mass", "flux_in", "flux_out", "max_u"):
        assert abs(d0[key] - d1[key]) <= 1e-12 * max(abs(d0[key]), 1e-300), key
    assert d1["time"] == steps and d1["n_nonfinite"] == 0
    whole.close()
    split.close()
    return u0


@pytest.mark.parametrize("n_parts", [2, 3])
def test_periodic_pipe_split_along_its_axis(n_parts):
    """Force-driven pipe with Bouzidi walls, periodic along z (the split axis): the first and
    last slabs exchange across the wrap."""
    g = I.pipe(16, 16, 48, 6.0, tau=0.6, g0=(0.0, 0.0, 1e-5), bouzidi=True)
    u = _compare(g, n_parts, 300)
    assert np.abs(u[2]).max() > 1e-4


@pytest.mark.parametrize("n_parts,storage,axis", [(2, "fp32", None), (3, "fp32", 0), (3, "fp32", 1), (2, "fp16", None)])
def test_aneurysm_split(n_parts, storage, axis):
    """The 64^3 synthetic aneurysm (Bouzidi walls, pulsatile inlet, outlet, absorbing layer),
    split along z (two slabs: the cut goes through the vessel, the sac and the relaxation-time
    field), along x (three slabs: cuts through the outlet segment and the sac) and along y
    (three slabs: through the inlet segment)."""
    g = I.aneurysm(2, edge=64, period=200.0, reynolds=30.0)
    plan = S.SlabPlan(g.mask.shape, g.periodic, n_parts, axis)
    assert len(plan.transfers(g.mask)) >= 2  # every case exchanges across at least one cut
    _compare(g, n_parts, 150, storage=storage, axis=axis)


def test_split_across_the_inlet_face():
    """A pipe along x with its inlet and outlet on the x faces, split along x: the end slabs hold
    the open boundaries, the middle slab none."""
    g = I.inlet_pipe(48, 12, 12, 4.7, u_peak=0.02, tau=0.6, bouzidi=True)
    g.wave = I.cardiac_waveform(3, period=150.0, u_peak=0.02)
    _compare(g, 3, 200, axis=0)


def test_split_after_init_equilibrium():
    """A periodic Taylor-Green box split in two along x, started from an equilibrium state: the
    exchange after the initialisation fills the halo layers."""
    rho0, u0 = I.taylor_green(32, 16, 8, 0.02)
    g = I.Geometry(mask=np.ones((8, 16, 32), np.uint8), periodic=(1, 1, 1), tau=0.7)
    _compare(g, 2, 60, init=(rho0, u0))


def _slab_rank(rank, world, port, steps, out):
    import os
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist

    from paper_2101_11107_gb300 import inputs as I2
    from paper_2101_11107_gb300 import lbm as L2
    from paper_2101_11107_gb300 import slabs as S2

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = I2.aneurysm(2, edge=48, period=200.0, reynolds=30.0)
        plan = S2.SlabPlan(g.mask.shape, g.periodic, world)
        dom = L2.Domain.from_geometry(plan.part_geometry(g, rank), scheme="ab")
        nv = plan.face_values()
        dev = torch.empty(nv, dtype=torch.int32, device="cuda")

        def pack(face, buf):  # device pack, then host copy for gloo
            dom.halo_pack(face, dev)
            buf.copy_(dev.cpu())

        def unpack(face, buf):
            dev.copy_(buf.cuda())
            dom.halo_unpack(face, dev)

        for _ in range(steps):
            dom.step(1)
            S2.exchange_between_ranks(plan, rank, pack, unpack, lambda: torch.empty(nv, dtype=torch.int32),
                                      mask=g.mask)
        rho, u = dom.macroscopic()
        sl = [slice(None)] * 3
        sl[2 - plan.axis] = plan.interior(rank)
        out[rank] = (plan.parts[rank].lo, plan.parts[rank].hi, u[(slice(None),) + tuple(sl)].tobytes())
        dom.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_through_gloo():
    """Two processes, one slab each (on the one GPU of this run), exchanging their face buffers
    through torch.distributed (gloo, host copies) after every step -- the path a run with one slab
    per GPU takes, with NCCL in place of gloo: the reassembled field equals the undivided domain's,
    bit for bit."""
    import socket

    import torch.multiprocessing as mp

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    steps = 60
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.start_processes(_slab_rank, args=(2, port, steps, out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    g = I.aneurysm(2, edge=48, period=200.0, reynolds=30.0)
    whole = lbm.Domain.from_geometry(g, scheme="ab")
    whole.step(steps)
    _, u0 = whole.macroscopic()
    whole.close()
    plan = S.SlabPlan(g.mask.shape, g.periodic, 2)
    for rank in range(2):
        lo, hi, buf = res[rank]
        shape = list(u0.shape)
        shape[3 - plan.axis] = hi - lo
        part = np.frombuffer(buf, dtype=np.float32).reshape(shape)
        sl = [slice(None)] * 4
        sl[3 - plan.axis] = slice(lo, hi)
        assert np.array_equal(part, u0[tuple(sl)]), rank
