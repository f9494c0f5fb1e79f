"""Storage precision on the Womersley pipe (radius 28 in a 64 x 64 x 256 box periodic along z,
tau 0.55, Womersley number 4, g_z(n) = 1e-5 cos(omega n)): FP32, FP16 and BF16 storage of the
populations (all arithmetic FP32) against the FP64 oracle and against the analytic Womersley
solution (the complex-Bessel profile of the oscillating pipe flow the paper's pulsatile cases
are characterised by, Sec. 2.2.2).

The oracle runs the one-layer z-slab (the flow is z-invariant: pinned on the oracle); the GPU
runs the full box and every z-layer is compared.  The study prints one JSON record per run
(``PRECISION_STUDY {...}``) with, per precision and sampled phase of the last period:
  rel_l2_oracle   ||u - u_oracle|| / ||u_oracle|| over the fluid cells,
  max_oracle      max |u - u_oracle| / max |u_oracle|,
  max_analytic    max |u - u_analytic| / (A / omega)  (A / omega: the inviscid velocity scale),
and the same for the oracle itself against the analytic solution (the discretisation error of
the halfway bounce-back staircase wall, common to every precision).

Errors are normalised by the period: the oscillating flow passes through rest twice a period,
where an error relative to the instantaneous field divides by almost nothing (the per-phase
numbers are reported too).  Bounds (asserted): FP32 stays within 1e-3 of the period's peak
velocity over ten periods (184,726 steps; measured 1.8e-4: the 1e-5 bar of the 1000-step parity
tests does not extend to this horizon); FP16 within 2e-2 relative L2 over the sampled phases; BF16 is reported only: the body force adds ~3e-5 per step to (f - w)/w ~ 5e-2,
below BF16's half-ulp of ~1e-4 there, so BF16 storage cannot represent this forcing (the same
stall as on the force-driven pipe).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2101_11107_gb300 import inputs as I

from . import analytic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_11107_gb300 import lbm  # noqa: E402

oracle.set_threads(min(16, os.cpu_count() or 1))


def _sample_times(period, periods, n_phases):
    """n_phases evenly spaced steps over the last of `periods` periods (rounded to integers)."""
    last = (periods - 1) * period
    return [int(round(last + (k + 1) * period / n_phases)) for k in range(n_phases)]


def run_study(storages, periods, n_phases):
    g = I.womersley_pipe()
    om, nu, A = g.gomega, g.info["nu"], g.gamp[2]
    period = 2.0 * math.pi / om
    times = _sample_times(period, periods, n_phases)
    fl = g.mask[0] > 0
    x = np.arange(g.mask.shape[2]) + 0.5
    X, Y = np.meshgrid(x, x)
    r = np.hypot(X - 32.0, Y - 32.0)
    R = g.info.get("radius", 28.0)
    scale = A / om

    ref = oracle.Case(g.mask[:1].copy(), periodic=g.periodic, tau=g.tau, gamp=g.gamp, gomega=om)
    ref_u = {}
    for t in times:
        ref.step(t - ref.time)
        ref_u[t] = ref.macroscopic()[1][2, 0]
    out = {"steps": times[-1], "periods": periods, "period_steps": period, "phases": n_phases, "A_over_omega": scale,
           "oracle_vs_analytic": [], "storage": {}}
    for t in times:
        ua = analytic.womersley(r, t, R, A, om, nu)
        out["oracle_vs_analytic"].append(float(np.abs(ref_u[t][fl] - ua[fl]).max() / scale))
    for storage in storages:
        dom = lbm.Domain.from_geometry(g, storage=storage)
        rows = []
        for t in times:
            dom.step(t - dom.time)
            rho, u = dom.macroscopic()
            uz = u[2]
            if storage == "fp32":  # z-invariance of the GPU run, bit for bit
                assert np.array_equal(uz, np.broadcast_to(uz[:1], uz.shape))
            ur = ref_u[t]
            du = uz[:, fl] - ur[fl][None, :]
            ua = analytic.womersley(r, t, R, A, om, nu)
            rows.append({"t": t,
                         "rel_l2_oracle": float(np.linalg.norm(du) / (np.linalg.norm(ur[fl]) * math.sqrt(uz.shape[0]))),
                         "max_oracle": float(np.abs(du).max() / np.abs(ur[fl]).max()),
                         "abs_max_oracle": float(np.abs(du).max()), "ref_max": float(np.abs(ur[fl]).max()),
                         "sq_err": float((du.astype(np.float64) ** 2).sum() / uz.shape[0]),
                         "sq_ref": float((ur[fl].astype(np.float64) ** 2).sum()),
                         "max_analytic": float(np.abs(uz[:, fl] - ua[fl][None, :]).max() / scale),
                         "finite": bool(np.all(np.isfinite(uz)))})
        dom.close()
        out["storage"][storage] = {
            # normalised by the period: the oscillating flow passes through rest twice a period,
            # where a per-phase relative error divides by a near-zero field
            "period_max_oracle": max(rw["abs_max_oracle"] for rw in rows) / max(rw["ref_max"] for rw in rows),
            "period_l2_oracle": math.sqrt(sum(rw["sq_err"] for rw in rows) / sum(rw["sq_ref"] for rw in rows)),
            "phase_rel_l2_oracle_max": max(rw["rel_l2_oracle"] for rw in rows),
            "phase_max_oracle_max": max(rw["max_oracle"] for rw in rows),
            "max_analytic": max(rw["max_analytic"] for rw in rows),
            "finite": all(rw["finite"] for rw in rows), "samples": rows}
    print("PRECISION_STUDY " + json.dumps(out), flush=True)
    return out


def test_womersley_fp16_one_period():
    """FP16 storage over the first period (18,472 steps): within 2e-2 relative L2 of the FP64
    oracle at 8 phases of the period."""
    res = run_study(["fp16"], periods=1, n_phases=8)
    s = res["storage"]["fp16"]
    assert s["finite"] and s["period_l2_oracle"] <= 2e-2 and s["phase_rel_l2_oracle_max"] <= 3e-2, s


def test_womersley_precision_study_ten_periods():
    """Ten periods (184,726 steps) in FP32, FP16 and BF16, sampled at 10 phases of the last
    period, against the oracle and the analytic solution."""
    res = run_study(["fp32", "fp16", "bf16"], periods=10, n_phases=10)
    st = res["storage"]
    # measured: 1.8e-4 (max) and 1.2e-4 (L2) of the peak velocity after 184,726 steps -- the
    # 1e-5 bar is met at 1000 steps (test_womersley_full_size_fp32); over this horizon the FP32
    # rounding of every step adds up to a small amplitude and phase offset, reported here and
    # held to a sanity bound 5x above it
    assert st["fp32"]["period_max_oracle"] <= 1e-3 and st["fp32"]["period_l2_oracle"] <= 1e-3, st["fp32"]
    assert st["fp16"]["finite"] and st["fp16"]["period_l2_oracle"] <= 2e-2, st["fp16"]
    assert st["bf16"]["finite"]
    # the FP32 run carries the discretisation error of the oracle and nothing more
    assert abs(st["fp32"]["max_analytic"] - max(res["oracle_vs_analytic"])) <= 1e-3
