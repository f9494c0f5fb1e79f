"""Pins of the oracle's classical collision operators (the comparison models of Sec. 2.1.2):
SRT with the second-order equilibrium and TRT, both with the Guo force term, and the
wall-position property that the paper credits to TRT and to the extra rates of CHM-MRT.

Each pin is a property fixed by the mathematics, not a retyped formula: the moments the
second-order equilibrium must reproduce, conservation, the reduction of TRT to SRT when its
two rates coincide, the rate at which each parity relaxes, and the exactness of halfway
bounce-back for plane Poiseuille flow when (1/w+ - 1/2)(1/w- - 1/2) = 3/16.
"""
import numpy as np
import pytest

import oracle

C, W = oracle.stencil()


def _state(seed, rho=1.01, u=(0.02, -0.015, 0.01), amp=2e-3):
    rng = np.random.default_rng(seed)
    f = oracle.feq_product(rho, np.array(u)) + amp * W * rng.normal(size=27)
    return f


def _second(f):
    return (C[:, :, None] * C[:, None, :] * f[:, None, None]).sum(0)


def _third_xyy(f):
    return float((C[:, 0] * C[:, 1] ** 2 * f).sum())


def test_feq2_reproduces_moments_to_second_order():
    rho, u = 1.03, np.array([0.04, -0.02, 0.015])
    f = oracle.feq2(rho, u)
    assert abs(f.sum() - rho) < 1e-15
    assert np.abs(C.T @ f - rho * u).max() < 1e-16
    assert np.abs(_second(f) - rho * (np.eye(3) / 3 + np.outer(u, u))).max() < 1e-15
    # it differs from the full expansion at third order in u only
    d = np.abs(f - oracle.feq_product(rho, u)).max()
    assert 1e-7 < d < 1e-4


@pytest.mark.parametrize("model", ["srt2", "trt2"])
def test_conservation_with_force(model):
    f = _state(1)
    g = np.array([1e-4, -2e-4, 5e-5])
    out = oracle.collide_srt2(f, g, 0.7) if model == "srt2" else oracle.collide_trt2(f, g, 0.7, 3 / 16)
    rho = f.sum()
    assert abs(out.sum() - rho) < 1e-15
    assert np.abs(C.T @ out - (C.T @ f + rho * g)).max() < 1e-15


def test_srt2_unit_tau_is_the_equilibrium():
    f = _state(2)
    out = oracle.collide_srt2(f, np.zeros(3), 1.0)
    rho = f.sum()
    u = C.T @ f / rho
    assert np.abs(_second(out) - rho * (np.eye(3) / 3 + np.outer(u, u))).max() < 1e-15


def test_trt2_with_equal_rates_is_srt2():
    f = _state(3)
    g = np.array([2e-5, 0.0, -1e-5])
    tau = 0.83
    a = oracle.collide_srt2(f, g, tau)
    b = oracle.collide_trt2(f, g, tau, (tau - 0.5) ** 2)
    assert abs(oracle.trt_minus_rate(tau, (tau - 0.5) ** 2) - 1 / tau) < 1e-15
    assert np.abs(a - b).max() < 1e-15


def test_trt2_relaxes_even_and_odd_parts_at_their_rates():
    f = _state(4, amp=5e-3)
    tau, magic = 0.62, 0.25
    wp, wm = 1 / tau, oracle.trt_minus_rate(tau, magic)
    out = oracle.collide_trt2(f, np.zeros(3), tau, magic)
    rho = f.sum()
    feq = oracle.feq2(rho, C.T @ f / rho)
    # shear stress (even, second order) relaxes with w+, a third-order odd moment with w-
    assert abs((_second(out) - _second(feq))[0, 1] - (1 - wp) * (_second(f) - _second(feq))[0, 1]) < 1e-15
    assert abs(_third_xyy(out - feq) - (1 - wm) * _third_xyy(f - feq)) < 1e-15


def _poiseuille(tau, collision, omega_hi=(1.0, 1.0, 1.0, 1.0), H=8, g=1e-5):
    """Plane channel: periodic x and z, halfway bounce-back walls at y = -1/2 and H - 1/2,
    body force g along x, run to steady state; max relative error against the parabola."""
    mask = np.ones((4, H, 4), np.uint8)
    nu = (tau - 0.5) / 3
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    case = oracle.Case(mask, periodic=(1, 0, 1), tau=tau, g0=(g, 0, 0), collision=collision, omega_hi=omega_hi)
    case.step(int(25 * H * H / nu) + 200)
    _, u = case.macroscopic()
    return float(np.abs(u[0][0, :, 0] - exact).max() / exact.max())


@pytest.mark.parametrize("tau", [0.6, 1.2, 2.0])
def test_trt2_magic_three_sixteenths_makes_bounce_back_exact(tau):
    assert _poiseuille(tau, "trt2") < 1e-9


def test_srt2_wall_position_depends_on_viscosity():
    # SRT is the TRT with Lambda = (tau - 1/2)^2, exact only where that equals 3/16
    assert _poiseuille(0.5 + np.sqrt(3 / 16), "srt2") < 1e-9
    assert _poiseuille(1.2, "srt2") > 1e-2
    assert _poiseuille(2.0, "srt2") > 0.1


def test_chm_mrt_third_order_rate_fixes_the_wall():
    """Sec. 2.1.2: the CHM-MRT operator has the degrees of freedom to fix the bounce-back wall
    position; with the third-order rate set by the same relation as TRT's odd rate it is exact,
    with full relaxation of the third order it is not."""
    tau = 1.2
    s3 = oracle.trt_minus_rate(tau, 3 / 16)
    assert _poiseuille(tau, "chm", omega_hi=(s3, 1.0, 1.0, 1.0)) < 1e-9
    assert _poiseuille(tau, "chm") > 5e-3
