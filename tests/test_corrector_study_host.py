"""Host-side helpers of the coarse-grid study (paper_2101_11107_gb300/corrector_study.py) that put
runs of different resolutions on one grid and find the resolution of equal error; CPU only."""
import numpy as np

from oracle import corrector as K
from paper_2101_11107_gb300 import corrector_study as S

rng = np.random.default_rng(5)


def test_sampling_at_twice_the_resolution_is_the_restriction():
    """e = 2 n: every coarse centre lies midway between its 8 children, so the fluid-weighted
    trilinear sample is the mean over the fluid children (the oracle's restriction)."""
    m = (rng.uniform(size=(8, 8, 8)) > 0.3).astype(np.uint8)
    u = rng.normal(size=(3, 8, 8, 8))
    got = S.sample_at_coarse_centres(u, m, 4)
    ref = K.restrict(u, m)
    has = K.restrict(np.ones((8, 8, 8)), m) > 0
    assert np.allclose(got[:, has], ref[:, has], rtol=1e-14, atol=1e-14)
    assert np.all(np.isnan(got[:, ~has]))


def test_sampling_at_the_same_resolution_is_the_identity():
    m = (rng.uniform(size=(6, 6, 6)) > 0.4).astype(np.uint8)
    u = rng.normal(size=(3, 6, 6, 6))
    got = S.sample_at_coarse_centres(u, m, 6)
    fl = m > 0
    assert np.array_equal(got[:, fl], u[:, fl]) and np.all(np.isnan(got[:, ~fl]))


def test_sampling_reproduces_a_linear_field():
    """A linear field on an all-fluid 12^3 grid sampled at the centres of an 8^3 grid of the same
    box (ratio 3/2) equals the field evaluated at those centres."""
    e, n = 12, 8
    x = np.arange(e) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.stack([0.3 * X - 0.1 * Y + 2.0, 0.2 * Z, -0.5 * X + 0.7 * Y + 0.1 * Z])
    got = S.sample_at_coarse_centres(u, np.ones((e, e, e), np.uint8), n)
    c = (np.arange(n) + 0.5) * e / n
    Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
    ref = np.stack([0.3 * Xc - 0.1 * Yc + 2.0, 0.2 * Zc, -0.5 * Xc + 0.7 * Yc + 0.1 * Zc])
    # centres within half a cell of the box edge clamp to the edge cells (no extrapolation)
    inner = (Xc > 0.5) & (Xc < e - 0.5) & (Yc > 0.5) & (Yc < e - 0.5) & (Zc > 0.5) & (Zc < e - 0.5)
    assert np.allclose(got[:, inner], ref[:, inner], rtol=0, atol=1e-12)


def test_rel_error_on_coarse_ignores_undefined_samples():
    m = np.ones((2, 2, 2), np.uint8)
    uf = np.ones((3, 2, 2, 2))
    ur = uf.copy()
    ur[0, 0, 0, 0] = np.nan
    ur[1, 1, 1, 1] = 1.5
    ok = np.ones((2, 2, 2), bool)
    ok[0, 0, 0] = False
    expect = 0.5 / np.linalg.norm(uf[:, ok])
    assert np.isclose(S.rel_error_on_coarse(ur, uf, m), expect)


def test_equal_error_point_hand_example():
    """Errors 0.20, 0.16, 0.10, 0 at edges 128, 160, 192, 256: 0.18 lies halfway between 128
    and 160, so e = 144; the wall time is interpolated in log-log between the two bracketing
    runs (1.0 s at 128, 2.0 s at 160)."""
    pt = S.equal_error_point([128, 160, 192, 256], [0.20, 0.16, 0.10, 0.0], [1.0, 2.0, 3.5, 8.0], 0.18)
    assert pt["between"] == [128, 160] and abs(pt["edge"] - 144.0) < 1e-12
    slope = np.log(2.0) / np.log(160 / 128)
    assert abs(pt["wall_s"] - np.exp(slope * np.log(144 / 128))) < 1e-12
    assert S.equal_error_point([128, 160], [0.20, 0.16], [1.0, 2.0], 0.25) is None
