"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports every entry point
declared in include/lbm.h, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2101_11107_gb300 import build as lib_build
from paper_2101_11107_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return lbm.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert set(declared_functions()) == set(lbm.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_default_params(L):
    p = lbm.Params()
    L.lbm_default_params(ctypes.byref(p))
    assert p.tau == 0.6 and list(p.omega_hi) == [1.0] * 4 and p.rho_out == 1.0 and p.storage == 0
    assert p.collision == 0 and p.trt_magic == 3.0 / 16.0


def _create(L, mask, links=None, params=None, inlet_center=None, inlet_radius=0.0):
    nz, ny, nx = mask.shape
    mask = np.ascontiguousarray(mask, np.uint8)
    p = lbm.Params()
    L.lbm_default_params(ctypes.byref(p))
    for k, v in (params or {}).items():
        if k == "periodic":
            for d in range(3):
                p.periodic[d] = v[d]
        else:
            setattr(p, k, v)
    if links is None:
        lc = ld = lq = None
        n = 0
    else:
        lc = np.ascontiguousarray(links[0], np.int64)
        ld = np.ascontiguousarray(links[1], np.uint8)
        lq = np.ascontiguousarray(links[2], np.float64)
        n = len(lc)
    ic = None if inlet_center is None else np.ascontiguousarray(inlet_center, np.float64)
    h = ctypes.c_void_p()
    st = L.lbm_create_domain(lbm._ptr(mask), nx, ny, nz, lbm._ptr(lc), lbm._ptr(ld), lbm._ptr(lq), n,
                             lbm._ptr(ic), inlet_radius, None, ctypes.byref(p), lbm.ALLOC_FN(0), lbm.FREE_FN(0),
                             None, None, ctypes.byref(h))
    return st, L.lbm_last_error().decode(), h


@pytest.mark.parametrize("case", ["mask_value", "periodic_extent", "tau", "tau_nan", "omega", "link_not_wall",
                                  "link_q", "link_q_nan", "link_q_above_one", "link_rest_direction",
                                  "link_on_inlet", "duplicate_link", "open_cell_off_face",
                                  "inlet_without_radius", "collision", "trt_magic", "halo_twist",
                                  "halo_inside", "halo_periodic_face", "link_into_halo"])
def test_invalid_arguments_rejected_before_device_work(L, case):
    mask = np.ones((4, 8, 8), np.uint8)
    mask[:, :, 0] = 0
    mask[:, :, -1] = 0
    kw = {}
    if case == "mask_value":
        mask[1, 1, 1] = 7
    elif case == "periodic_extent":
        mask = np.ones((6, 8, 8), np.uint8)
        kw["params"] = {"periodic": (1, 1, 1)}
    elif case == "tau":
        kw["params"] = {"tau": 0.5}
    elif case == "tau_nan":
        kw["params"] = {"tau": float("nan")}
    elif case == "omega":
        kw["params"] = {"omega_hi": (ctypes.c_double * 4)(1.0, 2.5, 1.0, 1.0)}
    elif case == "link_not_wall":
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [14], [0.3])  # +x neighbour of (1,2,1) is fluid
    elif case == "link_q":
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [12], [0.0])
    elif case == "link_q_nan":
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [12], [float("nan")])
    elif case == "link_q_above_one":
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [12], [1.5])
    elif case == "link_rest_direction":
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [13], [0.3])
    elif case == "link_on_inlet":
        mask[:, :, 1] = 2
        kw["links"] = ([1 + 8 * 2 + 64 * 1], [12], [0.3])
        kw["inlet_center"] = (0.0, 4.0, 2.0)
        kw["inlet_radius"] = 3.0
    elif case == "duplicate_link":
        kw["links"] = ([1 + 8 * 2 + 64 * 1] * 2, [12, 12], [0.3, 0.4])
    elif case == "open_cell_off_face":
        mask[2, 3, 3] = 3
    elif case == "inlet_without_radius":
        mask[:, :, 1] = 0
        mask[:, :, 0] = 2
    elif case == "collision":
        kw["params"] = {"collision": 3}
    elif case == "trt_magic":
        kw["params"] = {"collision": 2, "trt_magic": -1.0}
    elif case == "halo_twist":  # halo cells need the A-B scheme
        mask[0, 2:6, 1:7] = 4
    elif case == "halo_inside":  # a halo cell off every face
        mask[2, 3, 3] = 4
        kw["params"] = {"scheme": 0}
    elif case == "halo_periodic_face":  # z wraps: z = 0 is no face
        mask[0, 2:6, 1:7] = 4
        kw["params"] = {"scheme": 0, "periodic": (0, 0, 1)}
    elif case == "link_into_halo":  # a halo cell is fluid for its neighbours' links
        mask[0, :, 1:7] = 4
        kw["params"] = {"scheme": 0}
        kw["links"] = ([2 + 8 * 3 + 64 * 1], [4], [0.4])  # -z neighbour of (2,3,1) is a halo cell
    if case == "link_on_inlet":
        pass
    st, msg, h = _create(L, mask, **kw)
    assert st == 1, (case, st, msg)
    assert msg
    assert not h.value


def test_null_arguments(L):
    assert L.lbm_step(None, 1) == 1
    assert L.lbm_sync(None) == 1
    L.lbm_destroy(None)


def test_domain_beyond_the_32_bit_offset_range_is_rejected(L):
    """Kernels address populations with 32-bit offsets i * n_slots + slot: a 544^3 fully
    periodic box (161 M slots, 27 x slots > 2^32) must be refused before any device work."""
    mask = np.ones((544, 544, 544), np.uint8)
    st, msg, h = _create(L, mask, params={"periodic": (1, 1, 1)})
    assert st == 1 and "too large" in msg and not h.value


def test_batch_corrector_and_restriction_reject_invalid_arguments(L):
    """Entry points beyond the domain refuse bad arguments before any device work (INVALID_ARG,
    no handle written)."""
    out = ctypes.c_void_p(123)
    assert L.lbm_batch_create(None, 0, 10, None, ctypes.byref(out)) == 1 and not out.value
    members = (ctypes.c_void_p * 1)(None)
    out = ctypes.c_void_p(123)
    assert L.lbm_batch_create(members, 1, 0, None, ctypes.byref(out)) == 1  # graph_steps out of range
    assert "graph_steps" in L.lbm_last_error().decode() and not out.value
    out = ctypes.c_void_p(123)
    assert L.lbm_batch_create(members, 1, 10, None, ctypes.byref(out)) == 1  # NULL member
    assert not out.value

    assert L.lbm_corrector_num_params() == 3 * (27 * 16 * 16 + 16)
    params = np.zeros(L.lbm_corrector_num_params(), np.float32)

    def corrector(nx, ny, nz, scales=(0.05, 0.01, 0.005), alloc=None, free=None):
        mask = np.ones((nz, ny, nx), np.uint8)
        h = ctypes.c_void_p(123)
        st = L.lbm_corrector_create(lbm._ptr(mask), nx, ny, nz, *scales, lbm._ptr(params),
                                    alloc if alloc is not None else lbm.ALLOC_FN(0),
                                    free if free is not None else lbm.FREE_FN(0), None, None, ctypes.byref(h))
        return st, L.lbm_last_error().decode(), h

    st, msg, h = corrector(10, 8, 8)
    assert st == 1 and "multiples of 4" in msg and not h.value
    st, msg, h = corrector(8, 8, 8, scales=(0.05, 0.0, 0.005))
    assert st == 1 and "scales" in msg and not h.value
    st, msg, h = corrector(8, 8, 8, alloc=lbm.ALLOC_FN(lambda n, c: None))
    assert st == 1 and "allocator" in msg and not h.value

    buf = np.zeros(64, np.float32)
    fm = np.ones(64, np.uint8)
    assert L.lbm_restrict(lbm._ptr(buf), lbm._ptr(buf), lbm._ptr(fm), 3, 4, 4, lbm._ptr(buf), lbm._ptr(buf),
                          None) == 1
    assert L.lbm_restrict(None, lbm._ptr(buf), lbm._ptr(fm), 4, 4, 4, lbm._ptr(buf), lbm._ptr(buf), None) == 1


def test_autotune_cache_file(tmp_path):
    """The autotuner's JSON cache: a miss returns None (also for a missing or corrupt file), a
    stored entry comes back, a second key leaves the first in place, and the file is valid JSON
    after every write."""
    import json

    path = str(tmp_path / "tune.json")
    assert lbm.autotune_cache_get(path, "k1") is None
    lbm.autotune_cache_put(path, "k1", {"best": "128x6", "ms": {"128x6": 0.03}})
    assert lbm.autotune_cache_get(path, "k1")["best"] == "128x6"
    lbm.autotune_cache_put(path, "k2", {"best": "2c128x4", "ms": {}})
    data = json.load(open(path))
    assert set(data) == {"k1", "k2"} and data["k2"]["best"] == "2c128x4"
    open(path, "w").write("{not json")
    assert lbm.autotune_cache_get(path, "k1") is None
    lbm.autotune_cache_put(path, "k3", {"best": "128x7", "ms": {}})
    assert set(json.load(open(path))) == {"k3"}


def test_debug_variant_compiles(tmp_path):
    """The bounds-checked variant (-DLBM_DEBUG) of the step kernels and the host code compiles
    for sm_103a (the GPU test runs it)."""
    import subprocess

    src = os.path.join(ROOT, "paper_2101_11107_gb300", "csrc")
    for name in ("lbm_step_fp16.cu", "lbm_domain.cu"):
        cmd = [lib_build.NVCC, *lib_build.ARCH, *lib_build.FLAGS, "-DLBM_DEBUG", "-c", os.path.join(src, name),
               "-o", str(tmp_path / (name + ".o"))]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
