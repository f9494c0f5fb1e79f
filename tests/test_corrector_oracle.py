"""Pins of the corrector oracle (oracle/corrector.py): convolution identities, adjointness of
the two backward formulas, finite differences of the whole loss, restriction closed forms."""
import numpy as np
import pytest

from oracle import corrector as K
from paper_2101_11107_gb300 import inputs as I

rng = np.random.default_rng(99)


def test_conv_delta_and_shift_kernels():
    x = rng.normal(size=(16, 5, 6, 7))
    w = np.zeros((27, 16, 16))
    w[13] = np.eye(16)
    assert np.allclose(K.conv(x, w), x)
    w = np.zeros((27, 16, 16))
    o = 1 + 3 * 2 + 9 * 0  # (dx, dy, dz) = (0, +1, -1)
    w[o] = np.eye(16)
    y = K.conv(x, w)
    assert np.allclose(y[:, 1:, :-1, :], x[:, :-1, 1:, :])
    assert np.all(y[:, 0] == 0) and np.all(y[:, :, -1] == 0)


def test_backward_formulas_are_adjoints():
    """<conv(x, w), g> = <x, dX(g, w)> = <w, dW(g, x)> for random x, w, g."""
    x = rng.normal(size=(16, 4, 5, 6))
    w = rng.normal(size=(27, 16, 16))
    g = rng.normal(size=(16, 4, 5, 6))
    lhs = np.sum(K.conv(x, w) * g)
    assert abs(lhs - np.sum(x * K.conv_backward_input(g, w))) < 1e-9 * abs(lhs)
    assert abs(lhs - np.sum(w * K.conv_backward_weight(g, x))) < 1e-9 * abs(lhs)


def test_loss_gradient_matches_finite_differences():
    nz = ny = nx = 6
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.3).astype(np.uint8)
    rho = 1 + 0.01 * rng.normal(size=mask.shape)
    u = 0.03 * rng.normal(size=(3,) + mask.shape)
    x0 = K.features(rho, u, mask, 0.05, 0.01)
    params = I.corrector_init_params(3)
    params[1] = 0.05 * rng.normal(size=16)
    params[3] = 0.05 * rng.normal(size=16)
    target = rng.normal(size=(3,) + mask.shape)
    loss, grads = K.loss_and_grad(x0, target, mask, params)
    h = 1e-6
    for li, idx in [(0, (13, 2, 4)), (0, (0, 5, 1)), (1, (7,)), (2, (20, 3, 3)), (3, (0,)), (4, (13, 1, 8)),
                    (5, (2,)), (5, (10,))]:
        p2 = [q.copy() for q in params]
        p2[li][idx] += h
        lp, _ = K.loss_and_grad(x0, target, mask, p2)
        p2[li][idx] -= 2 * h
        lm, _ = K.loss_and_grad(x0, target, mask, p2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[li][idx]) < 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][idx])


def test_restriction_closed_forms():
    fm = np.ones((4, 4, 4), np.uint8)
    fm[0, 0, 0] = 0
    f = np.full((4, 4, 4), 2.5)
    f[0, 0, 0] = 1e9  # solid child: ignored
    c = K.restrict(f, fm)
    assert c.shape == (2, 2, 2) and np.allclose(c, 2.5)
    g = np.arange(64, dtype=float).reshape(4, 4, 4)
    c = K.restrict(g, np.ones((4, 4, 4)))
    assert np.isclose(c[1, 0, 1], g[2:4, 0:2, 2:4].mean())
    c = K.restrict(g, np.zeros((4, 4, 4)))
    assert np.all(c == 0)


def test_features_zero_at_solid():
    mask = np.zeros((3, 3, 3), np.uint8)
    mask[1, 1, 1] = 1
    x = K.features(np.full(mask.shape, 1.02), np.full((3,) + mask.shape, 0.01), mask, 0.05, 0.01)
    assert x[0, 1, 1, 1] == pytest.approx(0.2) and x[3, 1, 1, 1] == pytest.approx(2.0)
    assert np.count_nonzero(x[:, 0, 0, 0]) == 0 and np.all(x[5:] == 0) and x[4].sum() == 1


def _constant_output_params(b3):
    """Parameters whose network output is the constant b3 everywhere (W3 = 0)."""
    params = I.corrector_init_params(1)
    params[4] = np.zeros_like(params[4])
    params[5] = np.asarray(b3, dtype=np.float64)
    return params


def test_correction_clamps_the_network_output_not_du():
    """O = (5, -5, 0.5, ...) everywhere: with du_scale 0.005 and clip 2 the correction is
    (0.01, -0.01, 0.0025) at fluid cells and exactly 0 elsewhere.  A clamp applied to du instead
    of O (at +-2) would leave 0.025 and -0.025; a clamp on O alone with the wrong sign or a
    missing du_scale would give other values."""
    mask = np.zeros((4, 5, 6), np.uint8)
    mask[1:3, 1:4, 2:5] = 1
    b3 = np.zeros(16)
    b3[:3] = [5.0, -5.0, 0.5]
    x0 = K.features(np.ones(mask.shape), np.zeros((3,) + mask.shape), mask, 0.05, 0.01)
    du = K.correction(x0, mask, _constant_output_params(b3), 0.005)
    fl = mask > 0
    assert np.all(du[0][fl] == 0.005 * 2.0) and np.all(du[1][fl] == -0.005 * 2.0)
    assert np.allclose(du[2][fl], 0.005 * 0.5, rtol=0, atol=1e-18)
    assert np.all(du[:, ~fl] == 0.0)
    # inside the bounds the output passes unchanged: O = 1.999 -> du = 0.005 * 1.999
    b3[:3] = [1.999, -1.999, 0.0]
    du = K.correction(x0, mask, _constant_output_params(b3), 0.005)
    assert np.allclose(du[0][fl], 0.005 * 1.999, rtol=1e-15) and np.allclose(du[1][fl], -0.005 * 1.999, rtol=1e-15)
    assert np.all(du[2][fl] == 0.0)


def test_correction_keeps_a_non_finite_output_non_finite():
    """A network that has gone non-finite gives a non-finite correction at fluid cells (so that
    the corrected state is flagged and the plain solver takes over), and still 0 elsewhere."""
    mask = np.zeros((4, 4, 4), np.uint8)
    mask[1:3, 1:3, 1:3] = 1
    b3 = np.zeros(16)
    b3[0] = np.nan
    x0 = K.features(np.ones(mask.shape), np.zeros((3,) + mask.shape), mask, 0.05, 0.01)
    du = K.correction(x0, mask, _constant_output_params(b3), 0.005)
    fl = mask > 0
    assert np.all(np.isnan(du[0][fl])) and np.all(du[0][~fl] == 0.0) and np.all(du[1:] == 0.0)
