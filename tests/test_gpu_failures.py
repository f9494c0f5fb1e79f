"""Failure detection, driven from the host (nothing here faults, traps or hangs the GPU):

  * non-finite populations are reported as LBM_ERR_UNSTABLE by the FP64 diagnostics;
  * an allocator that returns NULL makes lbm_create_domain fail with LBM_ERR_OOM, leave *out
    NULL and give back every buffer it had obtained;
  * a learned corrector that has gone non-finite is caught and the coarse run falls back to the
    plain solver.
"""
import ctypes

import numpy as np
import pytest

from paper_2101_11107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402

UNSTABLE, OOM = 4, 3


def _diag(dom, name="lbm_get_diagnostics"):
    out = lbm.Diagnostics()
    st = getattr(lbm.load_library(), name)(dom._h, ctypes.byref(out))
    return st, out.as_dict()


@pytest.mark.parametrize("scheme", ["esoteric", "ab"])
def test_unstable_reported_for_a_non_finite_initial_state(scheme):
    """One fluid cell of a host density field holds a NaN: after lbm_init_equilibrium the
    diagnostics (both entry points) return UNSTABLE with the non-finite cells counted, the
    binding raises, and after a few steps the NaN has spread to more cells."""
    g = I.inlet_pipe(16, 12, 12, 4.5, u_peak=0.01, tau=0.7)
    dom = lbm.Domain.from_geometry(g, scheme=scheme)
    dom.step(3)
    assert _diag(dom)[0] == 0
    rho = np.ones(g.mask.shape, np.float32)
    u = np.zeros((3,) + g.mask.shape, np.float32)
    z, y, x = (int(v[0]) for v in np.nonzero(g.mask == 1))
    rho[z + 1, y + 2, x + 3] = np.nan
    assert g.mask[z + 1, y + 2, x + 3] == 1
    dom.init_equilibrium(rho, u)
    st, d = _diag(dom)
    assert st == UNSTABLE and d["n_nonfinite"] >= 1
    assert "non-finite" in lbm.load_library().lbm_last_error().decode()
    st2, d2 = _diag(dom, "lbm_get_diagnostics_noalloc")
    assert st2 == UNSTABLE and d2["n_nonfinite"] == d["n_nonfinite"]
    with pytest.raises(lbm.LbmError) as e:
        dom.diagnostics()
    assert e.value.status == UNSTABLE
    dom.step(4)
    st3, d3 = _diag(dom)
    assert st3 == UNSTABLE and d3["n_nonfinite"] > d["n_nonfinite"]


class CountingAllocator:
    """Torch-backed device allocator that returns NULL on its k-th call and counts what it hands
    out and gets back."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.freed = 0
        self.alloc_fn = lbm.ALLOC_FN(self._alloc)
        self.free_fn = lbm.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, ctx):
        assert ptr in self.live, "freed a pointer the allocator never handed out"
        del self.live[ptr]
        self.freed += 1


def _create(g, allocator, scheme):
    L = lbm.load_library()
    p = lbm.Params()
    L.lbm_default_params(ctypes.byref(p))
    p.tau = g.tau
    p.scheme = lbm.SCHEME[scheme]
    for d in range(3):
        p.periodic[d] = int(bool(g.periodic[d]))
    lc = np.ascontiguousarray(g.links[0], np.int64)
    ld = np.ascontiguousarray(g.links[1], np.uint8)
    lq = np.ascontiguousarray(g.links[2], np.float64)
    ic = np.ascontiguousarray(g.inlet_center, np.float64)
    mask = np.ascontiguousarray(g.mask, np.uint8)
    nz, ny, nx = mask.shape
    out = ctypes.c_void_p(12345)
    st = L.lbm_create_domain(lbm._ptr(mask), nx, ny, nz, lbm._ptr(lc), lbm._ptr(ld), lbm._ptr(lq), len(lc),
                             lbm._ptr(ic), float(g.inlet_radius), None, ctypes.byref(p), allocator.alloc_fn,
                             allocator.free_fn, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                             ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("scheme", ["esoteric", "ab"])
def test_create_domain_out_of_memory_at_every_allocation(scheme):
    """The allocator fails at its 1st, 2nd, ... call in turn: every failure gives OOM with a
    message, *out == NULL, and every buffer obtained before the failure is given back.  The
    first k that does not fail gives a working domain (all its allocations were exercised)."""
    g = I.inlet_pipe(16, 12, 12, 4.5, u_peak=0.01, tau=0.7, bouzidi=True)
    k = 1
    while True:
        a = CountingAllocator(k)
        st, out = _create(g, a, scheme)
        if st == 0:
            break
        assert st == OOM, (k, st)
        assert out.value is None, k
        assert "allocation failed" in lbm.load_library().lbm_last_error().decode()
        # everything handed out was given back (a failed call may be followed by the other
        # allocations of its group before the check)
        assert a.live == {} and a.freed == a.calls - 1, (k, a.calls, a.freed, len(a.live))
        k += 1
        assert k < 64
    assert k >= 12  # tables, populations, side buffer (twist), diagnostics
    lbm.load_library().lbm_step(out, 5)
    d = lbm.Diagnostics()
    assert lbm.load_library().lbm_get_diagnostics(out, ctypes.byref(d)) == 0 and d.n_nonfinite == 0
    n_held = len(a.live)
    lbm.load_library().lbm_destroy(out)
    assert a.live == {} and a.freed == n_held


def test_corrector_nan_output_propagates():
    """A non-finite network output gives a non-finite correction at fluid cells (the clamp lets
    NaN through), and exactly 0 at the other cells."""
    mask = np.zeros((16, 16, 16), np.uint8)
    mask[4:12, 4:12, 4:12] = 1
    params = I.corrector_init_params(1)
    params[5] = np.zeros(16)
    params[5][0] = np.nan
    net = lbm.Corrector(mask, params)
    rho = torch.ones(mask.shape, device="cuda")
    u = torch.zeros((3,) + mask.shape, device="cuda")
    du = net.forward(rho, u).cpu().numpy()
    fl = mask > 0
    assert np.all(np.isnan(du[0][fl])) and np.all(du[0][~fl] == 0)
    assert np.all(np.isfinite(du[1:]))


def test_corrector_fallback_to_plain_solver():
    """Host-set NaN parameters: the in-loop correction is detected as non-finite, the domain is
    put back to its state before the correction and the helper reports the fallback; the plain
    run then continues finite.  With finite parameters the correction is kept."""
    from paper_2101_11107_gb300 import corrector_study as S

    g = I.aneurysm(9, edge=64, period=200.0, reynolds=30.0)
    dom = lbm.Domain.from_geometry(g)
    dom.step(30)
    good = lbm.Corrector(g.mask, I.corrector_init_params(2))
    assert S.correct_or_fall_back(dom, good, None, None, 0.25) is True
    vec = good.params()
    vec[:] = np.nan
    bad = lbm.Corrector(g.mask, I.corrector_init_params(2))
    bad.set_params(vec)
    rho0, u0 = dom.macroscopic()
    assert S.correct_or_fall_back(dom, bad, None, None, 0.25) is False
    assert dom.diagnostics()["n_nonfinite"] == 0
    # the fallback re-initialises every population from the state before the correction: the
    # same fields, bit for bit, as a twin that never saw the bad network and is re-initialised
    # from the same rho, u
    twin = lbm.Domain.from_geometry(g)
    twin.step(30)
    assert S.correct_or_fall_back(twin, good, None, None, 0.25) is True
    twin.init_equilibrium(rho0, u0)
    assert all(np.array_equal(x, y) for x, y in zip(dom.macroscopic(), twin.macroscopic()))
    dom.step(40)
    twin.step(40)
    assert dom.diagnostics()["n_nonfinite"] == 0
    assert all(np.array_equal(x, y) for x, y in zip(dom.macroscopic(), twin.macroscopic()))
