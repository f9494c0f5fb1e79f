"""GPU parity of the classical collision operators the paper compares against (Sec. 2.1.2):
SRT and TRT with the second-order equilibrium and the Guo force term, selected by
lbm_params.collision, against the FP64 oracle's operators of the same name.

Tolerance: the FP32 bound of the CHM-MRT parity tests (max |u - u_ref| / max |u_ref| <= 1e-5,
|rho - rho_ref| <= 1e-5); the streaming, wall and open-boundary code is shared with CHM-MRT, so
these tests pin the collision kernels, their per-cell rates in an absorbing layer, and their
dispatch in every scheme and launch configuration.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2101_11107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402

oracle.set_threads(min(16, os.cpu_count() or 1))
TOL = 1e-5


def pair(g, steps, collision, scheme="esoteric", storage="fp32", magic=3.0 / 16.0, omega_hi=(1.0, 1.0, 1.0, 1.0)):
    dom = lbm.Domain.from_geometry(g, storage=storage, scheme=scheme, collision=collision, trt_magic=magic,
                                   omega_hi=omega_hi)
    ref = oracle.Case(g.mask, periodic=g.periodic, links=g.links, inlet_center=g.inlet_center,
                      inlet_radius=g.inlet_radius, tau=g.tau, g0=g.g0, gamp=g.gamp, gomega=g.gomega,
                      tau_cell=g.tau_cell, collision=collision, trt_magic=magic, omega_hi=omega_hi)
    if g.wave is not None:
        ref.set_waveform(*g.wave)
    dom.step(steps)
    ref.step(steps)
    rho, u = dom.macroscopic()
    rho_r, u_r = ref.macroscopic()
    dom.close()
    return rho, u, rho_r, u_r


def rel_u(u, u_r):
    return float(np.abs(u - u_r).max() / np.abs(u_r).max())


def _channel(tau, H=8, g=1e-5):
    mask = np.ones((4, H, 4), np.uint8)
    return I.Geometry(mask=mask, periodic=(1, 0, 1), tau=tau, g0=(g, 0.0, 0.0))


@pytest.mark.parametrize("collision,tau", [("trt2", 1.2), ("trt2", 0.6), ("srt2", 1.2)])
def test_plane_channel_to_steady_state(collision, tau):
    """Halfway bounce-back plane channel run to steady state: GPU against the oracle, and for
    TRT with Lambda = 3/16 against the exact parabola (the wall sits half-way for any tau)."""
    H, g0 = 8, 1e-5
    g = _channel(tau, H, g0)
    nu = (tau - 0.5) / 3
    steps = int(25 * H * H / nu) + 200
    rho, u, rho_r, u_r = pair(g, steps, collision)
    assert rel_u(u, u_r) <= TOL
    assert np.abs(rho - rho_r).max() <= 1e-5
    if collision == "trt2":
        y = np.arange(H)
        exact = g0 / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
        prof = u[0][:, :, :].mean(axis=(0, 2))
        assert np.abs(prof - exact).max() / exact.max() < 1e-4


def test_chm_mrt_with_magic_third_order_rate_on_gpu():
    """The CHM-MRT kernel with its third-order rate set from Lambda = 3/16 places the wall
    half-way too (Sec. 2.1.2): same check through the general (not second-order-only) path."""
    tau, H, g0 = 1.2, 8, 1e-5
    s3 = oracle.trt_minus_rate(tau, 3 / 16)
    g = _channel(tau, H, g0)
    nu = (tau - 0.5) / 3
    rho, u, rho_r, u_r = pair(g, int(25 * H * H / nu) + 200, "chm", omega_hi=(s3, 1.0, 1.0, 1.0))
    assert rel_u(u, u_r) <= TOL
    y = np.arange(H)
    exact = g0 / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert np.abs(u[0].mean(axis=(0, 2)) - exact).max() / exact.max() < 1e-4


@pytest.mark.parametrize("collision", ["srt2", "trt2"])
@pytest.mark.parametrize("scheme", ["esoteric", "ab"])
def test_bouzidi_pipe(collision, scheme):
    """Force-driven pipe with Bouzidi walls from rest, 1000 steps (the velocity grows
    throughout: a systematic FP32 momentum bias would show as a relative error growing in
    time, which the exact-momentum restoration of the kernel removes)."""
    g = I.pipe(16, 16, 8, 6.0, tau=0.6, g0=(0.0, 0.0, 1e-5), bouzidi=True)
    rho, u, rho_r, u_r = pair(g, 1000, collision, scheme=scheme)
    assert rel_u(u, u_r) <= TOL
    assert np.abs(rho - rho_r).max() <= 1e-5


@pytest.mark.parametrize("collision", ["srt2", "trt2"])
def test_open_boundaries(collision):
    g = I.inlet_pipe(16, 12, 12, 4.5, u_peak=0.01, tau=0.7)
    rho, u, rho_r, u_r = pair(g, 300, collision)
    assert rel_u(u, u_r) <= TOL
    assert np.abs(rho - rho_r).max() <= 1e-5


@pytest.mark.parametrize("collision", ["srt2", "trt2"])
def test_aneurysm_with_absorbing_layer(collision):
    """Bouzidi walls, pulsatile inlet, outlet, and per-cell relaxation times (the absorbing
    layer before the outlet: TRT derives each cell's odd rate from its own tau)."""
    g = I.aneurysm(1, edge=64, period=400.0, reynolds=20.0)
    assert g.tau_cell is not None
    rho, u, rho_r, u_r = pair(g, 300, collision)
    assert rel_u(u, u_r) <= TOL
    assert np.abs(rho - rho_r).max() <= 1e-5


@pytest.mark.parametrize("collision", ["srt2", "trt2"])
def test_schemes_and_launch_configs_agree_bitwise(collision):
    g = I.aneurysm(1, edge=64, period=400.0, reynolds=20.0)
    out = []
    for scheme, cfg in (("esoteric", 2), ("esoteric", 0), ("esoteric", 5), ("ab", 4)):
        d = lbm.Domain.from_geometry(g, scheme=scheme, collision=collision)
        d.set_launch_config(cfg)
        d.step(57)
        out.append(d.macroscopic())
        d.close()
    for rho, u in out[1:]:
        assert np.array_equal(rho, out[0][0]) and np.array_equal(u, out[0][1])


def test_fp16_storage_trt2():
    g = I.inlet_pipe(16, 12, 12, 4.5, u_peak=0.01, tau=0.7)
    rho, u, rho_r, u_r = pair(g, 300, "trt2", storage="fp16")
    assert np.linalg.norm(u - u_r) / np.linalg.norm(u_r) < 3e-3


def test_invalid_collision_rejected():
    g = _channel(0.8)
    with pytest.raises(Exception):
        lbm.Domain.from_geometry(g, collision=7)
    with pytest.raises(Exception):
        lbm.Domain.from_geometry(g, collision="trt2", trt_magic=0.0)


def test_srt_fails_where_chm_mrt_runs():
    """Sec. 2.1.2 / 3.4: at the small relaxation times of an under-resolved run the classical SRT
    operator with the second-order equilibrium becomes unstable while CHM-MRT keeps running.
    The synthetic aneurysm at Re 300 on a 64^3 and a 128^3 box (tau 0.5016 and 0.5032), one
    inflow period: SRT blows up (non-finite populations or max |u| > 0.35) on both, CHM-MRT on
    neither."""
    from paper_2101_11107_gb300 import stability_study as S

    res = S.run(edges=(64, 128), reynolds=300.0, seeds=(200,), periods=1.0, log=lambda m: None)
    for case in res["cases"]:
        assert case["chm"]["failed_at_step"] is None, case
        assert case["srt2"]["failed_at_step"] is not None, case
        assert case["chm"]["max_u"] < 0.2


def test_autotune_times_only_configurations_with_their_own_kernel():
    """The two-cell kernels exist for CHM-MRT at unit higher-order rates and the pipelined one
    for FP32 storage; elsewhere those configurations fall back and are reported as -1."""
    g = I.aneurysm(1, edge=64, period=400.0, reynolds=20.0)
    d = lbm.Domain.from_geometry(g, collision="srt2")
    best, ms = d.autotune(3)
    assert ms["2c128x4"] == -1 and ms["2c128x3"] == -1 and ms["pipe128x6"] > 0
    assert best not in (lbm.LAUNCH_CONFIG_NAMES.index("2c128x4"), lbm.LAUNCH_CONFIG_NAMES.index("2c128x3"))
    d.close()
    d = lbm.Domain.from_geometry(g, storage="fp16")
    best, ms = d.autotune(3)
    assert ms["pipe128x6"] == -1 and ms["2c128x4"] > 0
    d.close()
