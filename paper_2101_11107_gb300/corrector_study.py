"""Coarse grid + learned corrector versus the fine grid, on seeded synthetic aneurysms.

    python -m paper_2101_11107_gb300.corrector_study --out results.json            # full study
    python -m paper_2101_11107_gb300.corrector_study --small --out small.json      # quick check

Full study: fine 256^3 (tau from Re 300), coarse 128^3 with acoustic scaling (half the steps,
tau_c - 1/2 = (tau_f - 1/2)/2, the same lattice velocity and waveform over half the period:
Sec. 2.2.3 and 3.4 of the paper, 0.506 -> 0.503).  Training pairs come from the solver itself:
plain coarse states and the fine states restricted onto the coarse grid at the same physical
time, every 50 coarse steps of the last two periods of 32 seeded geometries (stored as
fluid-cell lists).  The trained network is evaluated two ways: as an output correction of the
plain coarse run (u_c + du at the sample times), and in the loop, nudging the coarse run every
50 steps with gain 1/4 after one period of warm-up (a full replacement every 50 steps, or nudges
in a feedback loop at gain 1/2, destabilise the coarse run at tau ~ 0.503), falling back to the
plain coarse solver if the state turns non-finite.  The corrector (3 conv layers, BF16 tensor cores) is trained on the
GPU and applied every 50 coarse steps after one period of warm-up.  Rounds of in-loop training
(DAgger-style: the states a running corrector is applied to, paired with the restricted fine
states at the same times, added to the training set) fit it to the states it meets in the
loop.  Evaluation on 8 held-out
geometries: relative L2 error of u against the restricted fine run over the coarse fluid cells
at 10 phases of the last cycle, the similarity index of the paper's Sec. 3.4 (read with the
factor 1/2 that bounds it by 1), and CUDA-event wall times of the fine, coarse and
coarse + corrector runs.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import json
import multiprocessing
import time

import numpy as np

U_SCALE, RHO_SCALE, DU_SCALE = 0.05, 0.01, 0.005


def _geometry_pair(args):
    from . import inputs as I

    seed, fine_edge, period_f, reynolds = args
    gf = I.aneurysm(seed, edge=fine_edge, period=period_f, wave_seed=seed, reynolds=reynolds)
    gc = I.aneurysm(seed, edge=fine_edge // 2, period=period_f / 2, wave_seed=seed, reynolds=reynolds)
    return seed, gf, gc


def geometry_pairs(seeds, fine_edge, period_f, reynolds, workers):
    """Generated on the host in parallel (spawned workers: no CUDA in them)."""
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        out = list(ex.map(_geometry_pair, [(s, fine_edge, period_f, reynolds) for s in seeds]))
    return {s: (gf, gc) for s, gf, gc in out}


def _geometry_at(args):
    from . import inputs as I

    seed, edge, period, reynolds = args
    return seed, edge, I.aneurysm(seed, edge=edge, period=period, wave_seed=seed, reynolds=reynolds)


def geometries_at_edges(seeds, edges, fine_edge, period_f, reynolds, workers):
    """The same seeded aneurysms at other resolutions (acoustic scaling: the period in steps and
    tau - 1/2 scale with the edge, the lattice velocity and Re stay); period_f * edge / fine_edge
    must be an integer."""
    jobs = []
    for s in seeds:
        for e in edges:
            period = period_f * e / fine_edge
            if period != int(period):
                raise ValueError(f"edge {e}: the period {period} is not a whole number of steps")
            jobs.append((s, e, int(period), reynolds))
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        out = list(ex.map(_geometry_at, jobs))
    return {(s, e): g for s, e, g in out}


def sample_at_coarse_centres(u, mask, n_coarse):
    """A velocity field u (3, e, e, e) on an e^3 grid sampled at the cell centres of the n_coarse^3
    grid of the same box: trilinear interpolation over the fluid cells of `mask` (the weights of
    non-fluid corners are dropped and the others renormalised), NaN where no corner is fluid.  For
    e = 2 n_coarse every centre lies midway between 8 children with equal weights, so this is the
    mean over the fluid children (the restriction of lbm_restrict); for e = n_coarse it is the
    identity; in between, the one operator puts runs of every resolution on the coarse grid."""
    e = mask.shape[0]
    fl = (mask > 0).astype(np.float64)
    idx, wts = [], []
    for _ in range(3):
        xc = (np.arange(n_coarse) + 0.5) * e / n_coarse - 0.5
        i0 = np.floor(xc).astype(np.int64)
        f = xc - i0
        i1 = np.minimum(i0 + 1, e - 1)
        idx.append((i0, i1))
        wts.append((1.0 - f, f))
    num = np.zeros((3, n_coarse, n_coarse, n_coarse))
    den = np.zeros((n_coarse, n_coarse, n_coarse))
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                zi, yi, xi = idx[2][bz], idx[1][by], idx[0][bx]
                w = wts[2][bz][:, None, None] * wts[1][by][None, :, None] * wts[0][bx][None, None, :]
                w = w * fl[np.ix_(zi, yi, xi)]
                den += w
                num += w[None] * u[(slice(None),) + np.ix_(zi, yi, xi)]
    out = np.full_like(num, np.nan)
    ok = den > 0
    out[:, ok] = num[:, ok] / den[ok]
    return out


def rel_error_on_coarse(u_run, u_fine, coarse_mask):
    """Relative L2 error of u_run against u_fine (both sampled on the coarse grid) over the
    coarse fluid cells where both are defined."""
    ok = (coarse_mask > 0) & np.all(np.isfinite(u_run), axis=0) & np.all(np.isfinite(u_fine), axis=0)
    return float(np.linalg.norm((u_run - u_fine)[:, ok]) / np.linalg.norm(u_fine[:, ok]))


def equal_error_point(edges, errors, walls, target):
    """The resolution at which the plain solver's error (decreasing with the edge) reaches
    `target`, by linear interpolation of the error in the edge between the two bracketing
    resolutions, and its wall time, by interpolation of log(wall) in log(edge).  None if the
    target lies outside the resolutions run."""
    pts = sorted(zip(edges, errors, walls))
    for (e0, r0, w0), (e1, r1, w1) in zip(pts[:-1], pts[1:]):
        if (r0 - target) * (r1 - target) <= 0 and r0 != r1:
            t = (r0 - target) / (r0 - r1)
            e = e0 + t * (e1 - e0)
            lw = np.log(w0) + (np.log(e) - np.log(e0)) / (np.log(e1) - np.log(e0)) * (np.log(w1) - np.log(w0))
            return {"edge": float(e), "wall_s": float(np.exp(lw)), "between": [e0, e1]}
    return None


def correct_or_fall_back(coarse, corrector, mask, out_mask, gain):
    """One in-loop correction of a running coarse domain, with the plain solver as fallback:
    the corrector nudges the domain's state; if the corrected state has a non-finite cell (FP64
    diagnostics count), the domain is put back to the macroscopic state it had before the
    correction (populations re-initialised at equilibrium from that rho and u) and False is
    returned, after which the caller runs the plain solver.  True: the correction was kept."""
    rho0, u0 = coarse.macroscopic_tensors()
    corrector.apply(coarse, mask=mask, out_mask=out_mask, gain=gain)
    if coarse.diagnostics(raise_unstable=False)["n_nonfinite"]:
        coarse.init_equilibrium(rho0, u0)
        return False
    return True


def similarity_index(u_hr, u_lr, mask):
    """Similarity index of Sec. 3.4 (factor 1/2) over the cells where mask != 0, computed on the
    device by lbm_similarity_index; u_hr, u_lr CUDA tensors (3, nz, ny, nx), mask a CUDA tensor."""
    from . import lbm

    return lbm.similarity_index(u_hr, u_lr, mask)


def run(fine_edge, period_f, reynolds, train_seeds, test_seeds, periods, samples_per_period, train_steps, lr,
        apply_every, workers, log, gain=0.25, dagger_rounds=0, dagger_steps=None, compare_edges=()):
    import torch

    from . import inputs as I
    from . import lbm

    t0 = time.time()
    pairs = geometry_pairs(list(train_seeds) + list(test_seeds), fine_edge, period_f, reynolds, workers)
    extra = geometries_at_edges(test_seeds, compare_edges, fine_edge, period_f, reynolds, workers) \
        if compare_edges else {}
    log(f"geometries: {len(pairs)} pairs and {len(extra)} at other resolutions in {time.time() - t0:.1f} s")
    torch.cuda.set_device(0)
    period_c = period_f // 2
    n_c = periods * period_c
    phase_step = period_c // samples_per_period
    sample_times = [n_c - period_c + k * phase_step for k in range(1, samples_per_period + 1)]
    # training also samples the period before the last
    train_times = sorted(set(sample_times) | {t - period_c for t in sample_times})
    assert all(t % apply_every == 0 for t in train_times)
    apply_from = period_c  # corrections start after one period of warm-up

    def tensors_mask(g):
        return torch.from_numpy(np.ascontiguousarray(g.mask > 0).astype(np.uint8)).cuda()

    def bulk_mask(g):
        """Fluid cells whose 26 neighbours are all fluid (cells outside the box count as solid):
        the cells the correction acts on."""
        fl = np.pad(g.mask > 0, 1)
        b = fl[1:-1, 1:-1, 1:-1].copy()
        nz, ny, nx = g.mask.shape
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    b &= fl[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        return torch.from_numpy(b.astype(np.uint8)).cuda()

    clip = 2.0 * DU_SCALE

    def simulate(gf, gc, corrector=None, times=None):
        """Fine, coarse (and optionally corrected coarse) runs over n_c coarse steps; returns the
        samples at `times` as dicts of CUDA tensors.  A corrected run that turns non-finite falls
        back to the plain coarse solver: it restarts from the last checked state and stops
        correcting (reported as 'fallback')."""
        times = sample_times if times is None else times
        fine = lbm.Domain.from_geometry(gf)
        coarse = lbm.Domain.from_geometry(gc)
        bf = lbm.Batch([fine], graph_steps=2 * apply_every)
        bc = lbm.Batch([coarse], graph_steps=apply_every)
        fmask = tensors_mask(gf)
        cmask = tensors_mask(gc)
        bmask = bulk_mask(gc)
        out = []
        state = {"fallback": None}
        for t in range(apply_every, n_c + 1, apply_every):
            bf.step(2 * apply_every)
            bc.step(apply_every)
            if corrector is not None and state["fallback"] is None and t >= apply_from:
                if not correct_or_fall_back(coarse, corrector, cmask, bmask, gain):
                    state["fallback"] = t
            if t in times:
                fr, fu = fine.macroscopic_tensors()
                cr, cu = lbm.restrict(fr, fu, fmask)
                rho, u = coarse.macroscopic_tensors()
                out.append({"t": t, "rho": rho, "u": u, "u_fine": cu, "rho_fine": cr})
        bf.close()
        bc.close()
        for d in (fine, coarse):
            if d.diagnostics(raise_unstable=False)["n_nonfinite"]:
                raise RuntimeError("the flow went unstable")
        if out:
            out[0]["fallback"] = state["fallback"]
        return out

    # ---------------------------------------------------------------- training data
    # plain fine and coarse runs side by side; every interval of the last two periods gives a
    # pair (coarse state, fine state restricted onto the coarse grid), stored as fluid-cell lists
    union = np.zeros(pairs[train_seeds[0]][1].mask.shape, bool)
    for s in pairs:
        union |= pairs[s][1].mask > 0
    masks, bulks, cells, data, fine_targets = {}, {}, {}, [], {}
    t1 = time.time()
    for s in train_seeds:
        gf, gc = pairs[s]
        masks[s] = tensors_mask(gc)
        bulks[s] = bulk_mask(gc)
        cells[s] = torch.nonzero(masks[s].reshape(-1)).reshape(-1)
        times = [t for t in range(apply_every, n_c + 1, apply_every) if t > n_c - 2 * period_c]
        for smp in simulate(gf, gc, times=times):
            idx = cells[s]
            fine_targets[(s, smp["t"])] = smp["u_fine"].reshape(3, -1)[:, idx].clone()
            data.append((s, smp["rho"].reshape(-1)[idx].clone(), smp["u"].reshape(3, -1)[:, idx].clone(),
                         fine_targets[(s, smp["t"])]))
    torch.cuda.synchronize()
    log(f"training data: {len(data)} samples from {len(train_seeds)} geometries in {time.time() - t1:.1f} s")
    shape = pairs[train_seeds[0]][1].mask.shape
    d_rho = torch.ones(shape, dtype=torch.float32, device="cuda")
    d_u = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    d_ut = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")

    def dense(sample):
        s, r, uu, ut = sample
        d_rho.fill_(1.0)
        d_u.zero_()
        d_ut.zero_()
        idx = cells[s]
        d_rho.view(-1)[idx] = r
        d_u.view(3, -1)[:, idx] = uu
        d_ut.view(3, -1)[:, idx] = ut
        return masks[s], bulks[s], d_rho, d_u, d_ut

    # ---------------------------------------------------------------- training
    net = lbm.Corrector(union.astype(np.uint8), I.corrector_init_params(0), U_SCALE, RHO_SCALE, DU_SCALE)
    rng = np.random.default_rng(0)
    losses = []

    def train(n_steps, lr0):
        for k in range(n_steps):
            m, bm, rho, u, ut = dense(data[rng.integers(len(data))])
            step_lr = lr0 if k < 0.7 * n_steps else lr0 * 0.2
            losses.append(net.train_step(rho, u, ut, step_lr, mask=m, out_mask=bm))
            if not np.isfinite(losses[-1]):
                raise RuntimeError(f"training diverged at step {k}")

    torch.cuda.synchronize()
    t2 = time.time()
    train(train_steps, lr)
    torch.cuda.synchronize()
    train_s = time.time() - t2
    log(f"training: {train_steps} steps in {train_s:.1f} s, loss {np.mean(losses[:50]):.4f} -> "
        f"{np.mean(losses[-50:]):.4f}")

    # ---------------------------------------------------------------- in-loop data (DAgger)
    # The network is applied to states of a coarse run that it has already been correcting,
    # which drift away from the plain coarse states it was trained on.  Each round runs the
    # coarse solver of every training geometry with the current network in the loop, pairs the
    # states it is applied to (before the correction) with the fine states restricted at the
    # same times (the fine run does not depend on the network), adds them to the training set
    # and trains on the union.
    def coarse_in_loop(gc, times):
        coarse = lbm.Domain.from_geometry(gc)
        bc = lbm.Batch([coarse], graph_steps=apply_every)
        cmask, bmask = tensors_mask(gc), bulk_mask(gc)
        out = {}
        for t in range(apply_every, n_c + 1, apply_every):
            bc.step(apply_every)
            if t in times:
                out[t] = coarse.macroscopic_tensors()
            if t >= apply_from:
                net.apply(coarse, mask=cmask, out_mask=bmask, gain=gain)
                if coarse.diagnostics(raise_unstable=False)["n_nonfinite"]:
                    out = None
                    break
        bc.close()
        return out

    dagger_log = []
    for rnd in range(dagger_rounds):
        t3 = time.time()
        added, unstable = 0, 0
        for s in train_seeds:
            states = coarse_in_loop(pairs[s][1], set(t for (s2, t) in fine_targets if s2 == s))
            if states is None:
                unstable += 1
                continue
            idx = cells[s]
            for t, (rho, u) in states.items():
                data.append((s, rho.reshape(-1)[idx].clone(), u.reshape(3, -1)[:, idx].clone(), fine_targets[(s, t)]))
                added += 1
        n_steps = dagger_steps if dagger_steps is not None else train_steps // 2
        train(n_steps, lr * 0.5)
        torch.cuda.synchronize()
        dagger_log.append({"round": rnd + 1, "added": added, "unstable_runs": unstable, "train_steps": n_steps,
                           "loss_last50": float(np.mean(losses[-50:])), "s": time.time() - t3})
        log(f"in-loop round {rnd + 1}: {added} samples added ({unstable} unstable runs), {n_steps} steps, "
            f"loss {np.mean(losses[-50:]):.4f}, {time.time() - t3:.1f} s")

    # ---------------------------------------------------------------- evaluation
    results = []
    for s in test_seeds:
        gf, gc = pairs[s]
        cm = gc.mask
        bm_eval = bulk_mask(gc)
        cm_eval = tensors_mask(gc)
        plain = simulate(gf, gc)
        corr = simulate(gf, gc, corrector=net)
        e_plain, e_corr, e_out, si_plain, si_corr, si_out = [], [], [], [], [], []
        fl = cm > 0
        for a, b in zip(plain, corr):
            uo_t = a["u"] + net.forward(a["rho"], a["u"], mask=cm_eval, out_mask=bm_eval)
            uf = a["u_fine"].cpu().numpy()
            up = a["u"].cpu().numpy()
            uc = b["u"].cpu().numpy()
            uo = uo_t.cpu().numpy()
            for arr, v in ((e_plain, up), (e_corr, uc), (e_out, uo)):
                arr.append(float(np.linalg.norm((v - uf)[:, fl]) / np.linalg.norm(uf[:, fl])))
            si_plain.append(similarity_index(a["u_fine"], a["u"], cm_eval))
            si_corr.append(similarity_index(a["u_fine"], b["u"], cm_eval))
            si_out.append(similarity_index(a["u_fine"], uo_t, cm_eval))
        # wall times, no sampling inside
        times = {}
        for name in ("fine", "coarse", "coarse+corrector"):
            g = gf if name == "fine" else gc
            dom = lbm.Domain.from_geometry(g)
            steps = 2 * n_c if name == "fine" else n_c
            chunk = 2 * apply_every if name == "fine" else apply_every
            b = lbm.Batch([dom], graph_steps=chunk)
            b.step(chunk)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for t in range(chunk, steps + 1, chunk):
                b.step(chunk)
                if name == "coarse+corrector" and t >= apply_from:
                    net.apply(dom, mask=cm_eval, out_mask=bm_eval, gain=gain)
            ev1.record()
            torch.cuda.synchronize()
            times[name] = ev0.elapsed_time(ev1) / 1e3
            b.close()
        # plain runs at intermediate resolutions, sampled on the coarse grid at the same physical
        # times, and timed like the others (for the comparison at equal error)
        plain_at = {}
        n_coarse = cm.shape[0]
        for e in compare_edges:
            ge = extra[(s, e)]
            errs = []
            dom = lbm.Domain.from_geometry(ge)
            for a in plain:
                te = a["t"] * e / n_coarse
                if te != int(te):
                    raise ValueError(f"edge {e}: sample time {te} is not a whole step")
                dom.step(int(te) - dom.time)
                ue = dom.macroscopic()[1].astype(np.float64)
                us = sample_at_coarse_centres(ue, ge.mask, n_coarse)
                errs.append(rel_error_on_coarse(us, a["u_fine"].cpu().numpy().astype(np.float64), cm))
            dom.close()
            steps_e = n_c * e // n_coarse
            dom = lbm.Domain.from_geometry(ge)
            b = lbm.Batch([dom], graph_steps=apply_every)
            b.step(apply_every)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            b.step(steps_e)
            ev1.record()
            torch.cuda.synchronize()
            plain_at[int(e)] = {"err": float(np.mean(errs)), "wall_s": ev0.elapsed_time(ev1) / 1e3,
                                "fluid": int(ge.nfluid), "steps": int(steps_e)}
            b.close()
            dom.close()
        # the plain coarse run through the same sampling operator (the identity at n_coarse)
        e_plain_resampled = []
        for a in plain:
            us = sample_at_coarse_centres(a["u"].cpu().numpy().astype(np.float64), cm, n_coarse)
            e_plain_resampled.append(rel_error_on_coarse(us, a["u_fine"].cpu().numpy().astype(np.float64), cm))
        r = {"seed": int(s), "fine_fluid": int(gf.nfluid), "coarse_fluid": int(gc.nfluid), "tau_fine": gf.tau,
             "tau_coarse": gc.tau, "err_plain": float(np.mean(e_plain)), "err_corrected": float(np.mean(e_corr)),
             "err_output_corrected": float(np.mean(e_out)),
             "err_plain_resampled": float(np.mean(e_plain_resampled)),
             "si_plain": float(np.mean(si_plain)), "si_corrected": float(np.mean(si_corr)),
             "si_output_corrected": float(np.mean(si_out)),
             "fallback_at_step": corr[0].get("fallback") if corr else None,
             "wall_s": times, "plain_at_edge": plain_at}
        log(json.dumps(r))
        results.append(r)
    summary = {
        "reynolds": reynolds, "fine_edge": fine_edge, "coarse_edge": fine_edge // 2, "period_fine": period_f, "periods": periods,
        "train_seeds": list(map(int, train_seeds)), "test_seeds": list(map(int, test_seeds)),
        "samples": len(data), "train_steps": train_steps, "train_s": train_s,
        "loss_first50": float(np.mean(losses[:50])), "loss_last50": float(np.mean(losses[-50:])),
        "apply_every": apply_every, "gain": gain, "dagger": dagger_log,
        "err_plain_mean": float(np.mean([r["err_plain"] for r in results])),
        "err_corrected_mean": float(np.mean([r["err_corrected"] for r in results])),
        "err_output_corrected_mean": float(np.mean([r["err_output_corrected"] for r in results])),
        "si_output_corrected_mean": float(np.mean([r["si_output_corrected"] for r in results])),
        "si_plain_mean": float(np.mean([r["si_plain"] for r in results])),
        "si_corrected_mean": float(np.mean([r["si_corrected"] for r in results])),
        "wall_fine_s": float(np.mean([r["wall_s"]["fine"] for r in results])),
        "wall_coarse_s": float(np.mean([r["wall_s"]["coarse"] for r in results])),
        "wall_coarse_corrector_s": float(np.mean([r["wall_s"]["coarse+corrector"] for r in results])),
        "per_geometry": results,
    }
    if compare_edges:
        # mean error and wall time of the plain solver against resolution (the coarse grid, the
        # intermediate grids, and the fine grid, whose error against itself is 0), and the
        # resolution and wall time at which it matches coarse + corrector's error
        edges = [fine_edge // 2] + [int(e) for e in compare_edges] + [fine_edge]
        errs = [summary["err_plain_mean"]] + \
            [float(np.mean([r["plain_at_edge"][int(e)]["err"] for r in results])) for e in compare_edges] + [0.0]
        walls = [summary["wall_coarse_s"]] + \
            [float(np.mean([r["plain_at_edge"][int(e)]["wall_s"] for r in results])) for e in compare_edges] + \
            [summary["wall_fine_s"]]
        pt = equal_error_point(edges, errs, walls, summary["err_corrected_mean"])
        summary["equal_error"] = {
            "edges": edges, "err_plain_by_edge": errs, "wall_plain_by_edge_s": walls,
            "target_err": summary["err_corrected_mean"], "plain_at_equal_error": pt,
            "wall_coarse_corrector_s": summary["wall_coarse_corrector_s"],
            "speedup_vs_plain_at_equal_error": (pt["wall_s"] / summary["wall_coarse_corrector_s"]) if pt else None,
            "speedup_vs_fine": summary["wall_fine_s"] / summary["wall_coarse_corrector_s"],
            "err_plain_resampled_mean": float(np.mean([r["err_plain_resampled"] for r in results]))}
    return summary, net


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--dagger", type=int, default=None,
                    help="rounds of in-loop data collection and training (default 4; --small: 2)")
    ap.add_argument("--gain", type=float, default=0.25)
    ap.add_argument("--compare-edges", default="",
                    help="comma-separated intermediate resolutions run plain for the comparison at equal error")
    a = ap.parse_args(argv)
    if a.small:
        cfg = dict(fine_edge=128, period_f=800, reynolds=60.0, train_seeds=list(range(100, 116)),
                   test_seeds=[200, 201], periods=3, samples_per_period=4, train_steps=1500, lr=2e-3, apply_every=50)
    else:
        cfg = dict(fine_edge=256, period_f=4000, reynolds=300.0, train_seeds=list(range(100, 132)),
                   test_seeds=list(range(200, 208)), periods=3, samples_per_period=10, train_steps=4000, lr=1e-3,
                   apply_every=50)
    dagger = a.dagger if a.dagger is not None else (2 if a.small else 4)
    edges = tuple(int(e) for e in a.compare_edges.split(",") if e)
    summary, net = run(workers=a.workers, log=lambda m: print(m, flush=True), dagger_rounds=dagger, gain=a.gain,
                       compare_edges=edges, **cfg)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(summary, f, indent=1)
    if a.weights:
        np.save(a.weights, net.params())
    print(json.dumps({k: v for k, v in summary.items() if k != "per_geometry"}), flush=True)


if __name__ == "__main__":
    main()
