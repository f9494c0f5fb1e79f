"""Pins of the oracle's single-node arithmetic against closed forms, invariants and special
cases fixed by the paper (Sec. 2.1.1, 2.1.3) and by the mathematics it relies on."""
import itertools
import math

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0
rng = np.random.default_rng(12345)


def rand_u(scale=0.15):
    return rng.uniform(-scale, scale, 3)


def test_stencil_isotropy():
    """D3Q27 weights: sum w = 1, sum w c_a c_b = cs^2 delta, fourth-order isotropy, and the
    weights factor into the D1Q3 weights (2/3, 1/6, 1/6)."""
    c, w = oracle.stencil()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(3), atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    for i in range(27):
        assert abs(w[i] - w1[c[i, 0]] * w1[c[i, 1]] * w1[c[i, 2]]) < 1e-16
        assert np.all(c[26 - i] == -c[i])


def test_hermite_tensor_closed_forms():
    """Grad's recurrence reproduces the textbook Hermite tensors up to fourth order."""
    x = rng.normal(size=3)
    H = oracle.hermite_tensor
    assert H([], x) == 1.0
    assert abs(H([1], x) - x[1]) < 1e-15
    assert abs(H([0, 0], x) - (x[0] ** 2 - CS2)) < 1e-14
    assert abs(H([0, 2], x) - x[0] * x[2]) < 1e-14
    assert abs(H([1, 1, 1], x) - (x[1] ** 3 - 3 * CS2 * x[1])) < 1e-14
    assert abs(H([0, 0, 1], x) - (x[0] ** 2 - CS2) * x[1]) < 1e-14
    assert abs(H([2, 2, 2, 2], x) - (x[2] ** 4 - 6 * CS2 * x[2] ** 2 + 3 * CS2 ** 2)) < 1e-13
    assert abs(H([0, 0, 1, 1], x) - (x[0] ** 2 - CS2) * (x[1] ** 2 - CS2)) < 1e-13
    # symmetric in its indices
    assert abs(H([0, 1, 0, 2], x) - H([2, 0, 0, 1], x)) < 1e-13


@pytest.mark.parametrize("trial", range(5))
def test_full_expansion_equals_product_form(trial):
    """Eq. (EDF) summed to the full D3Q27 expansion (Grad tensors, sixth order) equals the
    product form used by the solver."""
    u = rand_u(0.2)
    rho = rng.uniform(0.9, 1.1)
    a = oracle.feq_hermite(rho, u)
    b = oracle.feq_product(rho, u)
    assert np.max(np.abs(a - b)) < 2e-15


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_raw_moments_are_maxwellian(trial):
    """Every lattice-supported raw moment sum_i f_eq c_x^p c_y^q c_z^r (p,q,r <= 2) equals the
    Maxwellian's: prod_d mu_p(u_d) with mu = (1, u, u^2 + cs^2) times rho."""
    c, w = oracle.stencil()
    u = rand_u(0.2)
    rho = rng.uniform(0.9, 1.1)
    f = oracle.feq_product(rho, u)
    for p, q, r in itertools.product(range(3), repeat=3):
        mom = np.sum(f * c[:, 0] ** p * c[:, 1] ** q * c[:, 2] ** r)
        mu = [[1.0, ud, ud * ud + CS2] for ud in u]
        assert abs(mom - rho * mu[0][p] * mu[1][q] * mu[2][r]) < 1e-15


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_central_hermite_moments(trial):
    """Eq. (Hermite_coeff_eq): T f_eq = (rho, 0, ..., 0)."""
    u = rand_u(0.2)
    rho = rng.uniform(0.9, 1.1)
    a = oracle.chm_matrix(u) @ oracle.feq_product(rho, u)
    assert abs(a[0] - rho) < 1e-15
    assert np.max(np.abs(a[1:])) < 1e-15


def test_transform_is_central_hermite_tensor():
    """T[m][i] is the tensor Hermite polynomial of the index tuple x^p y^q z^r evaluated at the
    peculiar velocity c_i - u (Grad's recurrence, independent of the 1-D product)."""
    c, _ = oracle.stencil()
    u = rand_u()
    T = oracle.chm_matrix(u)
    for m in range(27):
        p, q, r = m % 3, (m // 3) % 3, m // 9
        idx = [0] * p + [1] * q + [2] * r
        for i in range(27):
            assert abs(T[m, i] - oracle.hermite_tensor(idx, c[i] - u)) < 1e-14


@pytest.mark.parametrize("trial", range(5))
def test_transform_round_trip(trial):
    """T^-1 (Kronecker of adjugate inverses) is the inverse of T: against numpy's general
    inverse, and T^-1 T f = f."""
    u = rand_u(0.2)
    T = oracle.chm_matrix(u)
    Ti = oracle.chm_inverse_matrix(u)
    assert np.max(np.abs(Ti - np.linalg.inv(T))) < 1e-13
    f = rng.uniform(0.0, 0.3, 27)
    assert np.max(np.abs(Ti @ (T @ f) - f)) < 1e-14


def near_eq(rho=None, u=None, noise=1e-3):
    u = rand_u(0.1) if u is None else u
    rho = rng.uniform(0.95, 1.05) if rho is None else rho
    return oracle.feq_product(rho, u) * (1.0 + noise * rng.normal(size=27))


@pytest.mark.parametrize("trial", range(5))
def test_collision_conserves_mass_and_momentum(trial):
    """Sec. 2.1.3: the CHM-MRT collision keeps rho and adds exactly the force F = rho g to the
    momentum."""
    c, _ = oracle.stencil()
    f = near_eq()
    g = rng.normal(size=3) * 1e-4
    s = oracle.rates(rng.uniform(0.51, 1.5), rng.uniform(0.5, 1.8, 4))
    fs = oracle.collide(f, g, s)
    rho = f.sum()
    assert abs(fs.sum() - rho) < 1e-15
    assert np.max(np.abs(c.T @ fs - (c.T @ f + rho * g))) < 1e-16


def test_single_rate_reduces_to_bgk():
    """S = I/tau on every moment turns T^-1 S T (f_eq - f) into (f_eq - f)/tau (Sec. 2.1.1)."""
    for _ in range(5):
        tau = rng.uniform(0.51, 2.0)
        f = near_eq(noise=1e-2)
        s = oracle.rates(tau, [1.0 / tau] * 4)
        assert np.max(np.abs(oracle.collide(f, np.zeros(3), s) - oracle.bgk(f, tau))) < 1e-15


def test_unit_rates_give_equilibrium():
    """S = I: f* = f_eq (every non-conserved moment set to its equilibrium value)."""
    f = near_eq(noise=1e-2)
    c, _ = oracle.stencil()
    rho = f.sum()
    u = c.T @ f / rho
    fs = oracle.collide(f, np.zeros(3), oracle.rates(1.0))
    assert np.max(np.abs(fs - oracle.feq_product(rho, u))) < 1e-15


def test_second_order_moments_relax_with_tau():
    """Post-collision second-order central Hermite moments equal (1 - 1/tau) times the
    pre-collision ones (a_eq = 0 there); third order with (1 - omega_3)."""
    tau = 0.7
    om = [1.3, 0.9, 1.1, 1.7]
    f = near_eq(noise=1e-2)
    c, _ = oracle.stencil()
    rho = f.sum()
    u = c.T @ f / rho
    T = oracle.chm_matrix(u)
    a = T @ f
    fs = oracle.collide(f, np.zeros(3), oracle.rates(tau, om))
    as_ = T @ fs
    for m in range(27):
        order = m % 3 + (m // 3) % 3 + m // 9
        if order == 2:
            assert abs(as_[m] - (1 - 1 / tau) * a[m]) < 1e-15
        if order >= 3:
            assert abs(as_[m] - (1 - om[order - 3]) * a[m]) < 1e-15


@pytest.mark.parametrize("axis,sign,inlet", [(0, 1, True), (1, -1, True), (2, 1, False), (0, -1, False)])
def test_open_boundary_postconditions(axis, sign, inlet):
    """Velocity inlet: sum f = rho with sum c f = rho u (u imposed); density outlet:
    sum f = rho_out, tangential momentum 0; known populations untouched."""
    c, _ = oracle.stencil()
    f = near_eq(noise=5e-3)
    u = np.zeros(3)
    u[axis] = sign * 0.03
    rho_out = 1.002
    g = oracle.zouhe(f, axis, sign, inlet, u, rho_out)
    known = c[:, axis] * sign <= 0
    assert np.all(g[known] == f[known])
    rho = g.sum()
    mom = c.T @ g
    if inlet:
        assert np.max(np.abs(mom - rho * u)) < 1e-15
    else:
        assert abs(rho - rho_out) < 1e-15
        t = [d for d in range(3) if d != axis]
        assert np.max(np.abs(mom[t])) < 1e-15


def test_waveform_normalisation():
    """U(t) = u_peak s(t)/max s: its maximum over a period is u_peak; a constant curve gives
    u_peak; the curve is periodic."""
    a = np.array([1.0, 0.3, -0.1, 0.05])
    b = np.array([0.2, 0.05, -0.02])
    P = 400.0
    vals = np.array([oracle.waveform(a, b, P, 0.05, t) for t in range(400)])
    assert abs(vals.max() - 0.05) < 1e-15
    assert abs(oracle.waveform(a, b, P, 0.05, 13.0) - oracle.waveform(a, b, P, 0.05, 413.0)) < 1e-15
    assert oracle.waveform(np.array([2.0]), np.zeros(0), 1.0, 0.03, 7.0) == pytest.approx(0.03, abs=1e-16)
