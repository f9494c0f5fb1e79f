"""The bounds-checked build (LBM_DEBUG): every access of the kernels is range-checked, and an
access out of range would be skipped and reported as LBM_ERR_STATE at the next synchronising
call.  On valid domains nothing may be reported, and the checks must not change a single bit:
the debug library runs the step kernels (esoteric twist and A-B, FP32 and FP16, Bouzidi walls,
open boundaries, absorbing layer), a batch, an equilibrium start and a velocity correction in a
child process and its fields are compared with the default library's."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2101_11107_gb300 import inputs as I
from paper_2101_11107_gb300 import lbm
out = {}
g = I.aneurysm(3, edge=64, period=200.0, reynolds=30.0)
for storage, scheme in (("fp32", "esoteric"), ("fp16", "ab"), ("fp32", "ab")):
    d = lbm.Domain.from_geometry(g, storage=storage, scheme=scheme)
    for cfg in (2, 6):
        d.set_launch_config(cfg)
        d.step(21)
    d.sync()
    rho, u = d.macroscopic()
    du = np.stack([0.001 * np.ones(g.mask.shape)] * 3).astype(np.float32) * (g.mask > 0)
    d.apply_velocity_correction(du)
    d.step(5)
    d.diagnostics()
    out[f"{storage}_{scheme}_u"] = u
    out[f"{storage}_{scheme}_u2"] = d.macroscopic()[1]
    d.close()
gs = [I.aneurysm(20 + k, edge=e, period=150.0, reynolds=40.0, wave_seed=50 + k) for k, e in enumerate((48, 64))]
ds = [lbm.Domain.from_geometry(x) for x in gs]
b = lbm.Batch(ds, graph_steps=10)
b.step(25)
for k, d in enumerate(ds):
    d.sync()
    out[f"batch{k}"] = d.macroscopic()[1]
b.close()
rho0, u0 = I.taylor_green(32, 16, 8, 0.02)
d = lbm.Domain(np.ones((8, 16, 32), np.uint8), periodic=(1, 1, 1), tau=0.7)
d.init_equilibrium(rho0, u0)
d.step(9)
d.sync()
out["tg"] = d.macroscopic()[1]
np.savez(sys.argv[2], **out)
print("ok", flush=True)
'''


def _run(lib, path):
    env = dict(os.environ)
    if lib:
        env["LBM_GB300_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, path], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
    return dict(np.load(path))


def test_debug_build_reports_nothing(tmp_path):
    """No check fires on valid domains (a reported fault raises in the child), and the fields
    agree with the default build: the fused step kernels, written with explicit roundings,
    bit for bit; the velocity correction, whose multiply-adds the compiler may contract
    differently around the added branches, within 1e-6 of max |u|."""
    from paper_2101_11107_gb300 import build as lib_build

    dbg = lib_build.build(debug=True)
    assert dbg != lib_build.LIB and os.path.exists(dbg)
    a = _run(dbg, str(tmp_path / "dbg.npz"))
    b = _run(None, str(tmp_path / "rel.npz"))
    assert set(a) == set(b)
    for k in a:
        if k.endswith("_u2"):
            assert np.abs(a[k] - b[k]).max() <= 1e-6 * np.abs(b[k]).max(), k
        else:
            assert np.array_equal(a[k], b[k]), k
