"""The seeded synthetic inputs follow their stated recipe (CPU only): box sizes, fluid counts,
relaxation times, Womersley number, waveform shape and the aneurysm's faces and wall links."""
import math

import numpy as np

from paper_2101_11107_gb300 import inputs as I


def test_direction_convention():
    """i = (cx+1) + 3(cy+1) + 9(cz+1), opposite 26 - i."""
    for i in range(27):
        cx, cy, cz = I.C27[i]
        assert i == (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)
        assert np.array_equal(I.C27[26 - i], -I.C27[i])


def test_poiseuille_pipe_recipe():
    """32x32x64, radius 12 along z through (16, 16), cell centres inside; tau 0.6, g 1e-6 along z,
    periodic along z: 448 fluid cells per slice."""
    g = I.poiseuille_pipe_32()
    assert g.mask.shape == (64, 32, 32)
    assert all(int(np.count_nonzero(g.mask[z])) == 448 for z in range(64))
    assert g.tau == 0.6 and tuple(g.g0) == (0.0, 0.0, 1e-6) and tuple(g.periodic)[2] == 1


def test_womersley_pipe_recipe():
    """64x64x256, radius 28, tau 0.55, body force 1e-5 cos(omega n) along z with Womersley
    number R sqrt(omega / nu) = 4: 2472 fluid cells per slice, 632,832 in all, period ~18,473."""
    g = I.womersley_pipe()
    assert g.mask.shape == (256, 64, 64)
    assert all(int(np.count_nonzero(g.mask[z])) == 2472 for z in range(0, 256, 37))
    assert g.nfluid == 632_832
    nu = (g.tau - 0.5) / 3.0
    assert g.tau == 0.55 and tuple(g.gamp) == (0.0, 0.0, 1e-5)
    assert abs(28.0 * math.sqrt(g.gomega / nu) - 4.0) < 1e-12
    assert round(2 * math.pi / g.gomega) == 18_473


def test_cardiac_waveform_recipe():
    """Five harmonics, a0 = 1, no backflow (min s >= 0.15 max s over the period), seeded."""
    for seed in range(8):
        a, b, period, u_peak = I.cardiac_waveform(seed)
        assert len(a) == 6 and len(b) == 5 and a[0] == 1.0 and period == 4000.0 and u_peak == 0.025
        t = np.arange(4000)
        k = np.arange(1, 6)
        ph = 2 * np.pi * np.outer(k, t) / period
        s = a[0] + (a[1:, None] * np.cos(ph) + b[:, None] * np.sin(ph)).sum(0)
        assert s.min() >= 0.15 * s.max()
        a2, b2, _, _ = I.cardiac_waveform(seed)
        assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert not np.array_equal(I.cardiac_waveform(0)[0], I.cardiac_waveform(1)[0])


def test_aneurysm_recipe():
    """Seeded aneurysm at edge 64 (lengths scaled by 64/256): vessel and sac radii in their
    ranges, inlet cells only on face y = 0 and outlet cells only on face x = 0, tau from Re 300
    on the peak mean velocity, Bouzidi links with q in (0, 1] from plain fluid cells into
    non-fluid neighbours, sorted and unique; the sponge raises tau by 0.1 at the outlet face;
    the same seed gives the same geometry."""
    edge, seed = 64, 7
    g = I.aneurysm(seed, edge=edge)
    par = I.aneurysm_params(seed, edge)
    s = edge / 256.0
    assert 10.0 * s <= par["r_vessel"] <= 14.0 * s and 20.0 * s <= par["r_sac"] <= 35.0 * s
    m = g.mask
    zz, yy, xx = np.nonzero(m == 2)
    assert len(yy) > 0 and np.all(yy == 0)
    zz, yy, xx = np.nonzero(m == 3)
    assert len(xx) > 0 and np.all(xx == 0)
    assert abs(g.tau - (0.5 + 3.0 * 0.025 * 2.0 * par["r_vessel"] / 300.0)) < 1e-15

    cell, beta, q = g.links
    assert len(cell) > 0
    assert np.all(q > 0.0) and np.all(q <= 1.0)
    nz, ny, nx = m.shape
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    assert np.all(m[z, y, x] == 1)
    c = I.C27[beta.astype(np.int64)]
    px, py, pz = x + c[:, 0], y + c[:, 1], z + c[:, 2]
    inside = (px >= 0) & (px < nx) & (py >= 0) & (py < ny) & (pz >= 0) & (pz < nz)
    assert not np.any(m[pz[inside], py[inside], px[inside]] != 0)
    key = cell * 27 + beta
    assert np.all(np.diff(key) > 0)
    assert np.all(beta != 13)

    assert abs(g.tau_cell[m == 3].max() - (g.tau + 0.1)) < 1e-12
    assert abs(g.tau_cell[:, :, edge // 2:].max() - g.tau) < 1e-15

    g2 = I.aneurysm(seed, edge=edge)
    assert np.array_equal(g.mask, g2.mask)
    assert all(np.array_equal(u, v) for u, v in zip(g.links, g2.links))
