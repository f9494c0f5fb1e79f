"""GPU flow metrics against the oracle: the similarity index kernel (lbm_similarity_index)
against oracle/metrics.py, running means (lbm_mean_*) against the mean of the oracle's
snapshots, and point probes (lbm_probe) against the exported fields and the oracle.

Tolerances: the similarity index is accumulated in FP64 from FP32 inputs on both sides, so the
two agree to rounding of the sums (1e-12); means and probes are FP32 fields held to the FP32
parity bound of the solver (1e-5 of the field maximum)."""
import os

import numpy as np
import pytest

import oracle
from oracle import metrics as M
from paper_2101_11107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402

oracle.set_threads(min(16, os.cpu_count() or 1))


@pytest.mark.parametrize("shape,frac", [((17, 33, 29), 0.6), ((64, 64, 64), 0.02), ((5, 1, 3), 1.0), ((300000,), 0.5)])
def test_similarity_index_matches_oracle(shape, frac):
    rng = np.random.default_rng(len(shape) * 7 + shape[0])
    ua = rng.normal(size=(3,) + shape).astype(np.float32)
    ub = (ua + 0.3 * rng.normal(size=ua.shape)).astype(np.float32)
    ub[:, rng.uniform(size=shape) < 0.05] = 0.0  # zero vectors
    mask = (rng.uniform(size=shape) < frac).astype(np.uint8)
    ta, tb, tm = torch.from_numpy(ua).cuda(), torch.from_numpy(ub).cuda(), torch.from_numpy(mask).cuda()
    si = lbm.similarity_index(ta, tb, tm)
    ref = M.similarity_index(ua, ub, mask)
    assert abs(si - ref) < 1e-12, (si, ref)
    assert lbm.similarity_index(ta, tb, tm) == si  # reproducible bit for bit
    assert abs(lbm.similarity_index(ta, ta) - 1.0) < 1e-12
    assert abs(lbm.similarity_index(ta, tb) - M.similarity_index(ua, ub, np.ones(shape))) < 1e-12


def test_similarity_index_empty_set_is_zero():
    u = torch.ones(3, 10, device="cuda")
    assert lbm.similarity_index(u, u, torch.zeros(10, dtype=torch.uint8, device="cuda")) == 0.0


def _pair(g):
    dom = lbm.Domain.from_geometry(g)
    ref = oracle.Case(g.mask, periodic=g.periodic, links=g.links, inlet_center=g.inlet_center,
                      inlet_radius=g.inlet_radius, tau=g.tau, g0=g.g0, tau_cell=g.tau_cell)
    if g.wave is not None:
        ref.set_waveform(*g.wave)
    return dom, ref


def test_running_means_match_oracle_snapshots():
    g = I.aneurysm(3, edge=64, period=300.0, reynolds=20.0)
    dom, ref = _pair(g)
    with pytest.raises(lbm.LbmError):
        dom.mean_sample()  # before reset: STATE
    dom.step(50)
    ref.step(50)
    dom.mean_reset()
    snaps_r, snaps_u = [], []
    for _ in range(12):
        dom.step(25)
        ref.step(25)
        dom.mean_sample()
        r, u = ref.macroscopic()
        snaps_r.append(r)
        snaps_u.append(u)
    rho_m, u_m, n = dom.mean()
    assert n == 12
    ur = M.time_mean(snaps_u)
    rr = M.time_mean(snaps_r)
    fl = g.mask > 0
    assert np.abs(u_m - ur)[:, fl].max() / np.abs(ur).max() <= 1e-5
    assert np.abs(rho_m - rr)[fl].max() <= 1e-5
    # compact export agrees with the dense one
    rc, uc, _ = dom.mean(dense=False)
    assert np.array_equal(rc, rho_m[fl]) and np.array_equal(uc, u_m[:, fl])
    dom.close()


def test_probes_match_fields_and_oracle():
    g = I.aneurysm(3, edge=64, period=300.0, reynolds=20.0)
    dom, ref = _pair(g)
    dom.step(120)
    ref.step(120)
    zyx = np.argwhere(g.mask > 0)
    pts = zyx[np.random.default_rng(0).choice(len(zyx), 40, replace=False)]
    out = dom.probe(pts)
    rho, u = dom.macroscopic()
    z, y, x = pts.T
    assert np.array_equal(out[:, 0], rho[z, y, x])
    assert np.array_equal(out[:, 1:].T, u[:, z, y, x])
    rr, ur = ref.macroscopic()
    assert np.abs(out[:, 1:].T - ur[:, z, y, x]).max() / np.abs(ur).max() <= 1e-5
    with pytest.raises(ValueError):
        dom.probe([[0, 0, 0]])  # a solid corner of the box
    idx = np.array([dom.info()["n_fluid"]], np.int64)
    assert lbm.load_library().lbm_probe(dom._h, lbm._ptr(idx), 1, lbm._ptr(np.empty(4, np.float32)), 0) == 1
    dom.close()
