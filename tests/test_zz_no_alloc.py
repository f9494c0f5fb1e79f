"""lbm_get_diagnostics_noalloc: the diagnostics reduction for callers that cannot allocate device
memory when they ask for it (a latency-bound monitoring loop, or an application whose device
memory another framework's pool already holds).  It runs with the library's fixed scratch array
and must give what lbm_get_diagnostics gives, call after call.

Collected last on purpose (file name), so that a run stopping at the first failure has run
every other test before this one; it also passes alone in a fresh process.
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

REL_TOL = 1e-12  # both calls run the same fixed-order FP64 reduction


def _via_abi(dom, name):
    out = lbm.Diagnostics()
    status = getattr(lbm.load_library(), name)(dom._h, ctypes.byref(out))
    return status, out.as_dict()


def _assert_same(a, b):
    for key in ("mass", "flux_in", "flux_out", "max_u"):
        assert abs(a[key] - b[key]) <= REL_TOL * max(abs(b[key]), 1e-300), (key, a[key], b[key])
    assert a["n_nonfinite"] == b["n_nonfinite"] and a["time"] == b["time"]


@pytest.mark.parametrize("storage,scheme", [("fp32", "esoteric"), ("fp16", "esoteric"), ("fp32", "ab")])
def test_noalloc_matches_allocating_reduction_twice(storage, scheme):
    g = I.aneurysm(6, edge=96, period=300.0, reynolds=30.0)
    dom = lbm.Domain.from_geometry(g, storage=storage, scheme=scheme)
    dom.step(40)
    st1, first = _via_abi(dom, "lbm_get_diagnostics_noalloc")
    st_ref, ref = _via_abi(dom, "lbm_get_diagnostics")
    assert st1 == 0 and st_ref == 0
    _assert_same(first, ref)
    assert first["flux_in"] > 0 and first["mass"] > 0
    # a second call in a row, after the state has moved on: no stale contents from the first
    dom.step(25)
    st2, second = _via_abi(dom, "lbm_get_diagnostics_noalloc")
    st_ref2, ref2 = _via_abi(dom, "lbm_get_diagnostics")
    assert st2 == 0 and st_ref2 == 0
    _assert_same(second, ref2)
    assert second["time"] == 65 and second["mass"] != first["mass"]


def test_noalloc_rejects_domains_beyond_its_scratch():
    """A domain with more than 2,097,152 fluid cells is refused with INVALID_ARG and a message,
    and nothing is launched."""
    mask = np.ones((128, 128, 132), np.uint8)  # 2,162,688 fluid cells
    dom = lbm.Domain(mask, periodic=(1, 1, 1), tau=0.8)
    status, _ = _via_abi(dom, "lbm_get_diagnostics_noalloc")
    assert status == 1
    assert "2097152" in lbm.load_library().lbm_last_error().decode()
    st, d = _via_abi(dom, "lbm_get_diagnostics")
    assert st == 0 and abs(d["mass"] - mask.size) < 1e-6


def test_noalloc_at_exactly_its_limit():
    """A fully fluid periodic 128^3 box has exactly 2,097,152 fluid cells, the largest domain the
    fixed scratch serves: the reduction then uses every partial-sum block of the array and the
    result record right after them.  Two calls in a row (the second after the flow has moved)
    must match the allocating reduction."""
    n = 128
    mask = np.ones((n, n, n), np.uint8)
    dom = lbm.Domain(mask, periodic=(1, 1, 1), tau=0.8, force=(1e-5, 0.0, 0.0))
    assert dom.info()["n_fluid"] == 2_097_152
    for _ in range(2):
        dom.step(3)
        st, got = _via_abi(dom, "lbm_get_diagnostics_noalloc")
        st_ref, ref = _via_abi(dom, "lbm_get_diagnostics")
        assert st == 0 and st_ref == 0
        _assert_same(got, ref)
        assert abs(got["mass"] - mask.size) < 1e-6 * mask.size and got["max_u"] > 0
