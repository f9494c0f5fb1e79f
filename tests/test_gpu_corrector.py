"""GPU parity of the learned corrector's kernels against the FP64 numpy oracle
(oracle/corrector.py) and of the velocity-correction step against the C oracle.

Tolerances: the network runs in BF16 (8 significant bits) with FP32 accumulation, so its output
at fluid cells is held to 2e-2 relative L2 of the FP64 result.  Gradients (BF16 activations and
output-gradients, FP32 accumulation) pick up one BF16 rounding of the back-propagated gradient
per layer they pass (dO, then dz2, then dz1), so the bound grows with depth: layer 3 cosine >=
0.999 and relative L2 <= 3e-2, layer 2 cosine >= 0.999 and relative L2 <= 5e-2, layer 1 cosine
>= 0.998 and relative L2 <= 8e-2 (the
layer-1 gradients are sums over thousands of cells with heavy cancellation, which magnifies the
relative effect of the per-element rounding).
Restriction and the velocity correction are FP32 and held to 1e-6 / 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import corrector as K
from paper_2101_11107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402

US, RS, DS = 0.05, 0.01, 0.005


def _case(n=16, seed=0):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    mask = (((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - 0.4 * n) ** 2) < (0.3 * n) ** 2).astype(np.uint8)
    mask[:, :, : n // 4] = 0
    rho = (1.0 + 0.01 * rng.normal(size=mask.shape)).astype(np.float32)
    u = (0.03 * rng.normal(size=(3,) + mask.shape)).astype(np.float32)
    ut = (u + 0.004 * rng.normal(size=u.shape)).astype(np.float32)
    params = I.corrector_init_params(seed)
    params[1] = (0.05 * rng.normal(size=16)).astype(np.float32).astype(np.float64)
    params[3] = (0.05 * rng.normal(size=16)).astype(np.float32).astype(np.float64)
    params[5] = (0.05 * rng.normal(size=16)).astype(np.float32).astype(np.float64)
    return mask, rho, u, ut, params


def _multi_slab_case(seed=0):
    """A 48 x 64 x 64 box (x, y, z) holding an ellipsoidal vessel with a cylindrical obstacle:
    1504 slabs of 8 x 16 x 1 cells (2688 active 4^3 tiles), so that every persistent CTA of the
    convolution (4 per SM) runs at least two slabs -- the double-buffered halo, both tensor
    memory accumulators and the mbarrier phase flips -- and so does every weight-gradient CTA
    (at most 304: both staging buffers, accumulators carried over slabs)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = 64, 64, 48
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    mask = ((((x - 24) / 23) ** 2 + ((y - 32) / 31) ** 2 + ((z - 32) / 31) ** 2) < 1).astype(np.uint8)
    mask[((x - 20) ** 2 + (y - 30) ** 2) < 36] = 0
    rho = (1.0 + 0.01 * rng.normal(size=mask.shape)).astype(np.float32)
    u = (0.03 * rng.normal(size=(3,) + mask.shape)).astype(np.float32)
    ut = (u + 0.004 * rng.normal(size=u.shape)).astype(np.float32)
    params = I.corrector_init_params(seed)
    for k in (1, 3, 5):
        params[k] = (0.05 * rng.normal(size=16)).astype(np.float32).astype(np.float64)
    return mask, rho, u, ut, params


def conv_work_counts(mask):
    """(slabs, tiles) the library evaluates for a creation mask: 4^3 tiles holding fluid, dilated
    by one tile, and the 8 x 16 x 1 slabs that meet them."""
    nz, ny, nx = mask.shape
    has = mask.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).any(axis=(1, 3, 5))
    p = np.pad(has, 1)
    use = np.zeros_like(has)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                use |= p[dz:dz + has.shape[0], dy:dy + has.shape[1], dx:dx + has.shape[2]]
    sl = use.reshape(use.shape[0], use.shape[1] // 4, 4, use.shape[2] // 2, 2).any(axis=(2, 4))
    return 4 * int(sl.sum()), int(use.sum())


def test_multi_slab_case_covers_every_cta_twice():
    mask = _multi_slab_case()[0]
    slabs, tiles = conv_work_counts(mask)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert slabs >= 2 * 4 * sms, (slabs, sms)
    assert slabs >= 2 * 304  # every weight-gradient CTA (at most 304) walks two or more slabs


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(seed):
    mask, rho, u, ut, params = _case(16, seed)
    net = lbm.Corrector(mask, params, US, RS, DS)
    du = net.forward(_t(rho), _t(u)).cpu().numpy()
    x0 = K.features(rho.astype(np.float64), u.astype(np.float64), mask, US, RS)
    ref = K.correction(x0, mask, params, DS)
    fl = mask > 0
    assert _rel(du[:, fl], ref[:, fl]) < 2e-2
    assert np.all(du[:, ~fl] == 0)


@pytest.mark.parametrize("seed", [0, 3])
def test_gradients_match_oracle(seed):
    mask, rho, u, ut, params = _case(16, seed)
    net = lbm.Corrector(mask, params, US, RS, DS)
    loss, grads = net.gradients(_t(rho), _t(u), _t(ut))
    x0 = K.features(rho.astype(np.float64), u.astype(np.float64), mask, US, RS)
    target = (ut.astype(np.float64) - u) / DS
    ref_loss, ref_grads = K.loss_and_grad(x0, target, mask, params)
    assert abs(loss - ref_loss) < 2e-2 * ref_loss
    bounds = {1: (0.998, 8e-2), 2: (0.999, 5e-2), 3: (0.999, 3e-2)}
    for name, g, r in zip(["W1", "b1", "W2", "b2", "W3", "b3"], grads, ref_grads):
        g, r = g.reshape(-1), r.reshape(-1)
        cos_min, rel_max = bounds[int(name[1])]
        cos = float(g @ r / (np.linalg.norm(g) * np.linalg.norm(r)))
        assert cos >= cos_min, (name, cos)
        assert _rel(g, r) <= rel_max, (name, _rel(g, r))


def test_forward_matches_oracle_multi_slab():
    """The forward pass where every convolution CTA walks two or more slabs."""
    mask, rho, u, ut, params = _multi_slab_case(0)
    net = lbm.Corrector(mask, params, US, RS, DS)
    du = net.forward(_t(rho), _t(u)).cpu().numpy()
    x0 = K.features(rho.astype(np.float64), u.astype(np.float64), mask, US, RS)
    ref = K.correction(x0, mask, params, DS)
    fl = mask > 0
    assert _rel(du[:, fl], ref[:, fl]) < 2e-2
    assert np.all(du[:, ~fl] == 0)


def test_gradients_match_oracle_multi_slab():
    """Loss and weight gradients where every convolution CTA (forward and data gradient) and
    every weight-gradient CTA walks two or more slabs (double-buffered staging, tensor-memory
    accumulators carried over slabs)."""
    mask, rho, u, ut, params = _multi_slab_case(1)
    net = lbm.Corrector(mask, params, US, RS, DS)
    loss, grads = net.gradients(_t(rho), _t(u), _t(ut))
    x0 = K.features(rho.astype(np.float64), u.astype(np.float64), mask, US, RS)
    target = (ut.astype(np.float64) - u) / DS
    ref_loss, ref_grads = K.loss_and_grad(x0, target, mask, params)
    assert abs(loss - ref_loss) < 2e-2 * ref_loss
    bounds = {1: (0.998, 8e-2), 2: (0.999, 5e-2), 3: (0.999, 3e-2)}
    for name, g, r in zip(["W1", "b1", "W2", "b2", "W3", "b3"], grads, ref_grads):
        g, r = g.reshape(-1), r.reshape(-1)
        cos_min, rel_max = bounds[int(name[1])]
        cos = float(g @ r / (np.linalg.norm(g) * np.linalg.norm(r)))
        print(name, f"cos {cos:.6f} rel {_rel(g, r):.3e}")
        assert cos >= cos_min, (name, cos)
        assert _rel(g, r) <= rel_max, (name, _rel(g, r))


def test_training_reduces_loss():
    """Adam on the GPU kernels fits a fixed synthetic correction (a smooth function of u):
    the loss falls at least tenfold in 300 steps."""
    mask, rho, u, _, params = _case(16, 5)
    ut = u.copy()
    ut[0] += 0.1 * u[1]
    ut[2] -= 0.05 * u[0]
    net = lbm.Corrector(mask, params, US, RS, DS)
    tr, tu, tt = _t(rho), _t(u), _t(ut)
    first = net.train_step(tr, tu, tt, 3e-3)
    for _ in range(300):
        last = net.train_step(tr, tu, tt, 3e-3)
    assert last < first / 10.0, (first, last)


def test_restriction_matches_oracle():
    rng = np.random.default_rng(4)
    fm = (rng.uniform(size=(8, 12, 16)) > 0.4).astype(np.uint8)
    fr = (1 + 0.01 * rng.normal(size=fm.shape)).astype(np.float32)
    fu = (0.02 * rng.normal(size=(3,) + fm.shape)).astype(np.float32)
    cr, cu = lbm.restrict(_t(fr), _t(fu), _t(fm))
    assert np.allclose(cr.cpu().numpy(), K.restrict(fr.astype(np.float64), fm), rtol=1e-6, atol=1e-7)
    assert np.allclose(cu.cpu().numpy(), K.restrict(fu.astype(np.float64), fm), rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("scheme", ["esoteric", "ab"])
def test_velocity_correction_matches_oracle(scheme):
    """Aneurysm (Bouzidi walls, inlet, outlet): 57 steps, a smooth synthetic du applied to the
    post-collision populations, 40 more steps; every cell against the oracle doing the same."""
    g = I.aneurysm(8, edge=64, period=200.0, reynolds=30.0)
    dom = lbm.Domain.from_geometry(g, scheme=scheme)
    ref = oracle.Case(g.mask, periodic=g.periodic, links=g.links, inlet_center=g.inlet_center,
                      inlet_radius=g.inlet_radius, tau=g.tau, tau_cell=g.tau_cell)
    ref.set_waveform(*g.wave)
    dom.step(57)
    ref.step(57)
    nz, ny, nx = g.mask.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    du = np.stack([0.002 * np.sin(x / 7.0), 0.001 * np.cos(y / 5.0), -0.0015 * np.sin(z / 9.0)])
    du = du.astype(np.float32) * (g.mask > 0)
    dom.apply_velocity_correction(du)
    ref.apply_velocity_correction(du.astype(np.float64))
    r0, u0 = dom.macroscopic()
    rr0, ur0 = ref.macroscopic()
    assert np.abs(u0 - ur0).max() / np.abs(ur0).max() <= 1e-5
    dom.step(40)
    ref.step(40)
    r1, u1 = dom.macroscopic()
    rr1, ur1 = ref.macroscopic()
    assert np.abs(u1 - ur1).max() / np.abs(ur1).max() <= 1e-5
    assert np.abs(r1 - rr1).max() <= 1e-5


def test_apply_through_corrector():
    """lbm_corrector_apply = export rho, u -> network -> velocity correction."""
    g = I.aneurysm(9, edge=64, period=200.0, reynolds=30.0)
    params = I.corrector_init_params(2)
    a = lbm.Domain.from_geometry(g)
    b = lbm.Domain.from_geometry(g)
    a.step(30)
    b.step(30)
    net = lbm.Corrector(g.mask, params, US, RS, DS)
    net.apply(a)  # creation mask, gain 1
    rho, u = b.macroscopic_tensors()
    b.apply_velocity_correction(net.forward(rho, u))
    assert np.array_equal(a.macroscopic()[1], b.macroscopic()[1])


def test_apply_with_the_domain_and_the_corrector_on_different_streams():
    """The domain's work on one stream, the corrector's on another: the apply orders the two
    (export -> network -> correction) and gives the same fields as with one stream."""
    import torch

    g = I.aneurysm(9, edge=64, period=200.0, reynolds=30.0)
    params = I.corrector_init_params(2)
    s_dom, s_net = torch.cuda.Stream(), torch.cuda.Stream()
    a = lbm.Domain.from_geometry(g, stream=s_dom)
    b = lbm.Domain.from_geometry(g)
    net_a = lbm.Corrector(g.mask, params, US, RS, DS, stream=s_net)
    net_b = lbm.Corrector(g.mask, params, US, RS, DS)
    for _ in range(3):
        a.step(20)
        b.step(20)
        net_a.apply(a, gain=0.5)
        net_b.apply(b, gain=0.5)
    assert np.array_equal(a.macroscopic()[1], b.macroscopic()[1])


def test_trained_corrector_gains_over_plain_coarse():
    """What the trained network gains over the method without it: the small study (fine 128^3 /
    coarse 64^3 synthetic aneurysms at Re 60, 16 training geometries, 2 held out), trained on the
    GPU by the corrector kernels.  On the held-out geometries the output-corrected coarse field
    is at least 5% closer (relative L2 of u against the restricted fine run) than the plain
    coarse field, the in-loop run (after two rounds of in-loop training) stays stable and is
    closer than the plain coarse run, and the coarse + corrector run is faster than the fine
    run."""
    from paper_2101_11107_gb300 import corrector_study as S

    summary, _ = S.run(fine_edge=128, period_f=800, reynolds=60.0, train_seeds=list(range(100, 116)),
                       test_seeds=[200, 201], periods=3, samples_per_period=4, train_steps=1500, lr=2e-3,
                       apply_every=50, workers=16, log=lambda m: None, dagger_rounds=2)
    assert summary["err_output_corrected_mean"] < 0.95 * summary["err_plain_mean"], summary
    assert summary["err_corrected_mean"] < summary["err_plain_mean"], summary
    assert all(r["fallback_at_step"] is None for r in summary["per_geometry"])
    assert summary["wall_coarse_corrector_s"] < summary["wall_fine_s"]


def test_training_is_reproducible():
    """The weight gradients are summed over the CTAs in a fixed order (no float atomics), so two
    training runs from the same parameters on the same samples end with the same parameters,
    bit for bit."""
    mask, rho, u, ut, params = _multi_slab_case(2)
    tr, tu, tt = _t(rho), _t(u), _t(ut)
    out = []
    for _ in range(2):
        net = lbm.Corrector(mask, params, US, RS, DS)
        for _ in range(20):
            net.train_step(tr, tu, tt, 1e-3)
        out.append(net.params())
        net.close()
    assert np.array_equal(out[0], out[1])


def test_apply_to_another_domain_matches_a_fresh_corrector():
    """The export inside lbm_corrector_apply clears the staging box only when it last held another
    domain: after an application to domain A, an application to domain B (another geometry in
    the same box) gives bit for bit what a fresh corrector gives on B, and so does a second one."""
    ga = I.aneurysm(9, edge=64, period=200.0, reynolds=30.0)
    gb = I.aneurysm(10, edge=64, period=200.0, reynolds=30.0)
    assert ((ga.mask > 0) & ~(gb.mask > 0)).any()  # cells that only A's export writes
    union = ((ga.mask > 0) | (gb.mask > 0)).astype(np.uint8)
    params = I.corrector_init_params(2)
    a = lbm.Domain.from_geometry(ga)
    b1 = lbm.Domain.from_geometry(gb)
    b2 = lbm.Domain.from_geometry(gb)
    for d in (a, b1, b2):
        d.step(30)
    used = lbm.Corrector(union, params, US, RS, DS)
    fresh = lbm.Corrector(union, params, US, RS, DS)
    used.apply(a)
    for _ in range(2):
        used.apply(b1, gain=0.5)
        fresh.apply(b2, gain=0.5)
        assert np.array_equal(b1.macroscopic()[1], b2.macroscopic()[1])
        b1.step(10)
        b2.step(10)
