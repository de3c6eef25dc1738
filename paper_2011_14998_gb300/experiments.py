"""Experiments of Section 3 on the synthetic workloads, built from the library's
entry points (no arithmetic of the method here, only bookkeeping and statistics).

* `adaptive_vs_dense` -- Section 3.2 (Figs. 7-9): the adaptive ray set
  (levels l_min -> l_max, 552 rays for 1 -> 4) against the dense set of level
  l_max (3072 rays for 4).  Each adaptive ray stands for the dense rays inside
  its pixel; its error is the relative difference between its u and the mean u
  of those dense rays, averaged over the bins above 1e-6 of the point's
  maximum.  Rays at l_max are dense rays themselves (error 0).
* `reduction_speedup` -- Table 2 (Section 3.2): original against reduced
  mesh, the reduction factor, the speed-up of the J solve and the error of the
  reduced J mapped back to the original points (Section 3.2.1).
* `batch_schedule` -- the batched persistent solve (one launch over many
  models) with its work list binned by traced length, longest first, against
  the same list in plain (model, origin, tile) order.
* `learned_vs_plain` -- the learned reduction against the plain criterion at
  one kept fraction: the network is trained on plain reductions of training
  seeds; the plain criterion's factors are scaled until it keeps the target
  fraction of the test mesh, and the network keeps as many points, either the
  top-ranked ones or by thinning weighted with its prediction.
* `batch_throughput`, `model_throughput` -- solves/s of one graph-replayed
  batched step over several models, and of the per-model entry point on one
  large model (the 10^6-particle spiral).

`python -m paper_2011_14998_gb300.experiments rays|reduction|learned|batch|batch64|octree|spiral` runs them
on the synthetic stand-ins and prints one JSON line each.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import MGX_FP32, MGX_FP64, mgx_antipode


def _dense_columns(rays_dense_row: np.ndarray, lmax: int) -> np.ndarray:
    """Column of the dense pair that contains each pixel of level lmax."""
    col = {int(r & 0x0FFFFFFF): c for c, r in enumerate(rays_dense_row)}
    npix = 12 * 4 ** lmax
    out = np.empty(npix, np.int64)
    for q in range(npix):
        out[q] = col[q] if q in col else col[mgx_antipode(lmax, q)]
    return out


def adaptive_vs_dense(ctx, m: dict, origins, l_min=1, l_max=4, precision=MGX_FP64, floor=1e-6):
    """Per-ray errors of the adaptive set against the dense set at the given origins."""
    mid_a = ctx.load(m, l_min=l_min, l_max=l_max)
    mid_d = ctx.load(m, l_min=l_max, l_max=l_max)
    try:
        ra, rd = ctx.rays(mid_a), ctx.rays(mid_d)
        cols = _dense_columns(rd[0], l_max)
        errs, levels, ja, jd = [], [], [], []
        for o in origins:
            ua = ctx.solve_u(mid_a, int(o), int(o) + 1, precision=precision)[0]
            ud = ctx.solve_u(mid_d, int(o), int(o) + 1, precision=precision)[0]
            lev = (ra[o] >> 28).astype(np.int64)
            pix = (ra[o] & 0x0FFFFFFF).astype(np.int64)
            wa = 2.0 / (12.0 * 4.0 ** lev)
            ja.append((wa[:, None] * ua).sum(0))
            jd.append((2.0 / (12.0 * 4.0 ** l_max)) * ud.sum(0))
            mask = ja[-1] > floor * ja[-1].max()
            for p in range(len(pix)):
                k = 4 ** (l_max - lev[p])
                desc = pix[p] * k + np.arange(k)
                ref = ud[cols[desc]].mean(0)
                rel = np.abs(ua[p] - ref)[mask] / np.abs(ref[mask])
                errs.append(rel.mean())
                levels.append(lev[p])
        errs, levels = np.array(errs), np.array(levels)
        ja, jd = np.array(ja), np.array(jd)
        mj = jd > floor * jd.max(axis=1, keepdims=True)
        return dict(n_origins=len(origins), rays_adaptive=2 * ra.shape[1], rays_dense=2 * rd.shape[1],
                    frac_rays_below_10pct=float((errs < 0.1).mean()), frac_rays_below_20pct=float((errs < 0.2).mean()),
                    frac_rays_below_1e3=float((errs < 1e-3).mean()),
                    frac_rays_at_finest_level=float((levels == l_max).mean()),
                    max_err_finest_level=float(errs[levels == l_max].max()) if (levels == l_max).any() else 0.0,
                    median_ray_err=float(np.median(errs)),
                    J_rel_err_mean=float((np.abs(ja - jd)[mj] / jd[mj]).mean()),
                    J_rel_err_max=float((np.abs(ja - jd)[mj] / jd[mj]).max()))
    finally:
        ctx.free(mid_a)
        ctx.free(mid_d)


def reduction_speedup(ctx, m: dict, f_small, f_large, G_thres, seed=1, precision=MGX_FP32, reps=3):
    """Plain reduction of m, solve times on both meshes and the reduced-mesh error (Table 2 shape)."""
    import torch

    from . import learned

    def timed_solve(model):
        mid = ctx.load(model)
        ctx.solve_J(mid, precision=precision)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            J = ctx.solve_J(mid, precision=precision)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        return mid, J, dt

    mid, J_full, t_full = timed_solve(m)
    keep = ctx.reduce_mesh(mid, m["rho"], f_small, f_large, G_thres, seed)[3]
    ctx.free(mid)
    r = learned.remesh(m, keep)
    mid_r, J_red, t_red = timed_solve(r)
    ctx.free(mid_r)
    err = learned.point_errors(J_full, learned.interpolate(r["pos"], J_red, m["pos"]))
    return dict(n_original=len(m["pos"]), n_reduced=len(r["pos"]), reduction=len(m["pos"]) / len(r["pos"]),
                t_full_s=t_full, t_reduced_s=t_red, speedup=t_full / t_red, mean_rel_err=float(err.mean()),
                p90_rel_err=float(np.quantile(err, 0.9)), frac_below_1pct=float((err < 0.01).mean()),
                frac_below_10pct=float((err < 0.1).mean()))


def error_cdf(err: np.ndarray, bins: int = 1000, lo: float = -8.0, hi: float = 1.0):
    """Cumulative distribution of per-point relative errors over `bins` bins
    uniform in log10(error) on [lo, hi] (errors below 10^lo in the first bin):
    (bin upper edges, fraction of points at or below each edge)."""
    e = np.log10(np.maximum(np.asarray(err, np.float64), 10.0 ** lo))
    edges = np.linspace(lo, hi, bins + 1)[1:]
    h = np.histogram(np.minimum(e, hi), bins=bins, range=(lo, hi))[0]
    return edges, np.cumsum(h) / max(len(e), 1)


def reduction_sweep(ctx, m: dict, table1, scales=(1.0, 1.4, 2.0), seed=1, precision=MGX_FP32, reps=3,
                    std=None, alpha=2.0):
    """Solve-time speed-up against reduction factor (Table 2 shape, Fig. 6): the
    plain criterion with Table 1's factors scaled by each of `scales`, and, when
    a trained network's feature standardiser `std` is given, the weighted learned
    thinning at the same kept fraction.  Per run: reduction factor, speed-up of
    the reduced solve, mean and p90 per-point error, and its CDF (1000 bins)."""
    import torch

    from . import learned

    def timed_solve(model):
        mid = ctx.load(model)
        ctx.solve_J(mid, precision=precision)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            J = ctx.solve_J(mid, precision=precision)
        torch.cuda.synchronize()
        return mid, J, (time.perf_counter() - t0) / reps

    f_small, f_large, g_thres = table1
    mid, J_full, t_full = timed_solve(m)
    runs = []
    try:
        for k in scales:
            keeps = {"plain": ctx.reduce_mesh(mid, m["rho"], f_small * k, f_large * k, g_thres, seed)[3]}
            if std is not None:
                keeps["learned_weighted"] = learned.reduce_learned_weighted(ctx, mid, m, std,
                                                                            float(keeps["plain"].mean()), alpha, seed)
            for crit, keep in keeps.items():
                r = learned.remesh(m, keep)
                mr, J_red, t_red = timed_solve(r)
                ctx.free(mr)
                err = learned.point_errors(J_full, learned.interpolate(r["pos"], J_red, m["pos"]))
                edges, cdf = error_cdf(err)
                runs.append(dict(criterion=crit, scale=k, n_reduced=len(r["pos"]),
                                 reduction=len(m["pos"]) / len(r["pos"]), t_reduced_s=t_red,
                                 speedup=t_full / t_red, mean_rel_err=float(err.mean()),
                                 p90_rel_err=float(np.quantile(err, 0.9)), cdf_log10_edges=edges.tolist(),
                                 cdf=cdf.tolist()))
    finally:
        ctx.free(mid)
    return dict(n_original=len(m["pos"]), t_full_s=t_full, runs=runs)


def batch_schedule(ctx, models, precision=MGX_FP32, reps=3):
    """Step time of one batched solve over `models` with the cost-binned and the plain work list."""
    import torch

    from . import MGX_BATCH_GRAPH, MGX_BATCH_RAYS

    mids = [ctx.load(m) for m in models]
    saved = ctx.tuning()
    out = dict(n_models=len(models), points=int(sum(len(m["pos"]) for m in models)))
    try:
        solves = 0
        for mid, m in zip(mids, models):
            solves += ctx.models[mid]["n"] * ctx.models[mid]["npairs"] * ctx.models[mid]["L"] * ctx.models[mid]["F"]
        out["solves_per_step"] = int(solves)
        outs = None
        for name, sched in (("binned", 0), ("plain", 1)):
            ctx.set_tuning(dict(saved, schedule=sched))
            flags = MGX_BATCH_GRAPH | MGX_BATCH_RAYS
            outs = ctx.solve_J_batch(mids, precision=precision, outs=outs, flags=flags)
            ctx.solve_J_batch(mids, precision=precision, outs=outs, flags=flags)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                ctx.solve_J_batch(mids, precision=precision, outs=outs, flags=flags)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            out[f"step_s_{name}"] = dt
            out[f"solves_per_s_{name}"] = solves / dt
        out["binned_speedup"] = out["step_s_plain"] / out["step_s_binned"]
    finally:
        ctx.set_tuning(saved)
        for k in mids:
            ctx.free(k)
    return out


def batch_throughput(ctx, models, precision=MGX_FP32, reps=1):
    """Aggregate solves/s of one graph-replayed batched step over all `models`
    (one persistent launch), with the planning and first eager step timed apart."""
    import torch

    from . import MGX_BATCH_GRAPH, MGX_BATCH_RAYS

    mids = [ctx.load(m) for m in models]
    try:
        solves = sum(ctx.models[k]["n"] * ctx.models[k]["npairs"] * ctx.models[k]["L"] * ctx.models[k]["F"]
                     for k in mids)
        flags = MGX_BATCH_GRAPH | MGX_BATCH_RAYS
        t0 = time.perf_counter()
        outs = ctx.solve_J_batch(mids, precision=precision, flags=flags)  # plan, eager step, capture
        torch.cuda.synchronize()
        t_plan = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.solve_J_batch(mids, precision=precision, outs=outs, flags=flags)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        ok = all(bool(torch.isfinite(o).all()) for o in outs)
    finally:
        for k in mids:
            ctx.free(k)
    return dict(n_models=len(models), points=int(sum(len(m["pos"]) for m in models)), solves_per_step=int(solves),
                plan_and_first_step_s=t_plan, step_s=dt, solves_per_s=solves / dt, all_finite=ok)


def model_throughput(ctx, m, precision=MGX_FP32, reps=2):
    """Solves/s of the per-model entry point (mgx_solve_J traces and solves the
    origins in chunks that fit its arena) on one model, J left on the device;
    the ingest with its ray set and the first solve are timed apart."""
    import torch

    t0 = time.perf_counter()
    mid = ctx.load(m)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t0
    try:
        i = ctx.models[mid]
        solves = i["n"] * i["npairs"] * i["L"] * i["F"]
        out = torch.empty((i["n"], i["L"] * i["F"]), dtype=torch.float64, device=f"cuda:{ctx.device}")
        t0 = time.perf_counter()
        ctx.solve_J(mid, precision=precision, out=out)
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.solve_J(mid, precision=precision, out=out)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        ok = bool(torch.isfinite(out).all())
        ctx.profile(True)  # one more step, untimed, for the work counters and the kernel split
        ctx.solve_J(mid, precision=precision, out=out)
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
    finally:
        ctx.free(mid)
    return dict(points=int(i["n"]), pairs=int(i["npairs"]), solves_per_step=int(solves), load_s=t_load,
                first_step_s=t_first, step_s=dt, solves_per_s=solves / dt, all_finite=ok,
                samples_per_solve=prof["samples"] / solves, updates_per_solve=prof["updates"] / solves,
                trace_points_per_half=prof["trace_points"] / (i["n"] * i["npairs"] * 2),
                samples_per_s=prof["samples"] / dt, kernel_ms=prof["ms"])


def learned_vs_plain(ctx, make_model, train_seeds, test_seed, table1, keep_fraction=0.2,
                     scales=(1.0, 1.5, 2.2), epochs=60, seed=11):
    """Reduced-mesh error of the learned and the plain criterion at one kept fraction."""
    from . import learned

    f_small, f_large, g_thres = table1
    Xs, ys = [], []
    for s_ in train_seeds:
        m = make_model(s_)
        reds = [(f_small * k, f_large * k, g_thres, 1000 + 10 * s_ + j) for j, k in enumerate(scales)]
        X, y = learned.training_samples(ctx, m, reds)
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    std, losses, _ = learned.train_network(ctx, X, y, epochs=epochs, seed=1)
    test = make_model(test_seed)
    mid = ctx.load(test)
    try:
        J_full = ctx.solve_J(mid, precision=MGX_FP32)
        lo, hi = 0.25, 16.0  # scale of both factors; the kept fraction falls as it grows
        for _ in range(40):
            k = np.sqrt(lo * hi)
            keep = ctx.reduce_mesh(mid, test["rho"], f_small * k, f_large * k, g_thres, seed)[3]
            if keep.mean() > keep_fraction:
                lo = k
            else:
                hi = k
            if hi / lo < 1.001:
                break
        keep_plain = ctx.reduce_mesh(mid, test["rho"], f_small * hi, f_large * hi, g_thres, seed)[3]
        keep_mlp = learned.reduce_learned(ctx, mid, test, std, float(keep_plain.mean()))
        keep_w = {a: learned.reduce_learned_weighted(ctx, mid, test, std, float(keep_plain.mean()), a, seed)
                  for a in (0.5, 1.0, 2.0, 3.0)}
    finally:
        ctx.free(mid)
    e_plain = learned.reduction_error(ctx, test, J_full, keep_plain)
    e_mlp = learned.reduction_error(ctx, test, J_full, keep_mlp)
    weighted = {}
    for a, kw in keep_w.items():
        e = learned.reduction_error(ctx, test, J_full, kw)
        weighted[f"alpha_{a}"] = dict(kept_fraction=float(kw.mean()), mean_rel_err=float(e.mean()),
                                      p90=float(np.quantile(e, 0.9)))
    return dict(n=len(test["pos"]), kept_fraction=float(keep_plain.mean()),
                reduction=float(1.0 / keep_plain.mean()), plain_scale=float(hi), train_samples=int(len(y)),
                loss_first=float(losses[0]), loss_last=float(losses[-1]),
                mean_rel_err_plain=float(e_plain.mean()), mean_rel_err_learned=float(e_mlp.mean()),
                p90_plain=float(np.quantile(e_plain, 0.9)), p90_learned=float(np.quantile(e_mlp, 0.9)),
                frac_below_1pct_plain=float((e_plain < 0.01).mean()),
                frac_below_1pct_learned=float((e_mlp < 0.01).mean()), weighted=weighted)


def learned_reduction_study(ctx, make_train, train_seeds, test_model, table1, fractions=(0.2, 0.1),
                            scales=(1.0, 1.5, 2.2), alphas=(1.0, 2.0), epochs=40, seed=11):
    """Train the reduction network once on J errors of plain reductions of the
    training models, then compare the plain criterion, the top-ranked points and
    the weighted thinning at each kept fraction of the test model (same number
    of points kept): mean and p90 of the per-point J error after re-meshing and
    barycentric interpolation back to the full mesh."""
    from . import learned

    f_small, f_large, g_thres = table1
    t0 = time.perf_counter()
    Xs, ys = [], []
    for s_ in train_seeds:
        m = make_train(s_)
        reds = [(f_small * k, f_large * k, g_thres, 1000 + 10 * s_ + j) for j, k in enumerate(scales)]
        X, y = learned.training_samples(ctx, m, reds)
        Xs.append(X)
        ys.append(y)
        del m
    X, y = np.concatenate(Xs), np.concatenate(ys)
    std, losses, _ = learned.train_network(ctx, X, y, epochs=epochs, seed=1)
    t_train = time.perf_counter() - t0
    test = test_model
    mid = ctx.load(test)
    rows = []
    try:
        J_full = ctx.solve_J(mid, precision=MGX_FP32)
        for frac in fractions:
            lo, hi = 0.25, 16.0
            for _ in range(40):
                k = np.sqrt(lo * hi)
                keep = ctx.reduce_mesh(mid, test["rho"], f_small * k, f_large * k, g_thres, seed)[3]
                if keep.mean() > frac:
                    lo = k
                else:
                    hi = k
                if hi / lo < 1.001:
                    break
            keeps = {"plain": ctx.reduce_mesh(mid, test["rho"], f_small * hi, f_large * hi, g_thres, seed)[3]}
            kf = float(keeps["plain"].mean())
            keeps["top_k"] = learned.reduce_learned(ctx, mid, test, std, kf)
            for a in alphas:
                keeps[f"weighted_alpha_{a}"] = learned.reduce_learned_weighted(ctx, mid, test, std, kf, a, seed)
            for name, kp in keeps.items():
                e = learned.reduction_error(ctx, test, J_full, kp)
                rows.append(dict(target_fraction=frac, criterion=name, kept_fraction=float(kp.mean()),
                                 reduction=float(1.0 / kp.mean()), mean_rel_err=float(e.mean()),
                                 p90=float(np.quantile(e, 0.9)), frac_below_1pct=float((e < 0.01).mean())))
    finally:
        ctx.free(mid)
    return dict(n_test=len(test["pos"]), train_seeds=list(train_seeds), train_samples=int(len(y)),
                train_s=t_train, loss_first=float(losses[0]), loss_last=float(losses[-1]), rows=rows)


def main(argv):
    import synth

    from . import Context, build

    build()
    ctx = Context(0)
    try:
        which = argv[1] if len(argv) > 1 else "rays"
        if which == "rays":
            m = synth.wind_model(int(argv[2]) if len(argv) > 2 else 50000, seed=2, n_freq=50)
            o = np.sort(np.random.default_rng(0).choice(len(m["pos"]), 200, replace=False))
            print(json.dumps(dict(experiment="adaptive_vs_dense", workload=m["name"],
                                  **adaptive_vs_dense(ctx, m, o))), flush=True)
        elif which == "batch":
            k = int(argv[2]) if len(argv) > 2 else 16
            models = synth.batch_models(n_models=k, seed=5, n_min=10_000, n_max=50_000, n_lines=2, n_freq=50)
            print(json.dumps(dict(experiment="batch_schedule", lines=2, bins_per_line=50, rays="adaptive l 0-3",
                                  **batch_schedule(ctx, models))), flush=True)
        elif which == "octree":
            n = int(argv[2]) if len(argv) > 2 else 300_000
            t0 = time.perf_counter()
            m = synth.octree_model(n, seed=3)
            gen = time.perf_counter() - t0
            print(json.dumps(dict(experiment="batch_throughput", workload=m["name"], lines=2, bins_per_line=64,
                                  rays="adaptive l 0-3", generation_s=gen,
                                  **batch_throughput(ctx, [m], reps=3))), flush=True)
        elif which == "spiral":
            n = int(argv[2]) if len(argv) > 2 else 1_000_000
            t0 = time.perf_counter()
            m = synth.spiral_model(n, seed=4)
            gen = time.perf_counter() - t0
            print(json.dumps(dict(experiment="model_throughput", workload=m["name"], lines=1, bins_per_line=100,
                                  rays="l = 2 (96 pairs)", generation_s=gen, **model_throughput(ctx, m))), flush=True)
            print(json.dumps(dict(experiment="batch_throughput", workload=m["name"], lines=1, bins_per_line=100,
                                  rays="l = 2 (96 pairs)", **batch_throughput(ctx, [m], reps=2))), flush=True)
        elif which == "batch64":
            n_max = int(argv[2]) if len(argv) > 2 else 200_000
            t0 = time.perf_counter()
            models = synth.batch_models(n_models=64, seed=5, n_min=10_000, n_max=n_max, n_lines=4, n_freq=100)
            gen = time.perf_counter() - t0
            print(json.dumps(dict(experiment="batch_throughput", n_max=n_max, lines=4, bins_per_line=100,
                                  rays="adaptive l 0-3", generation_s=gen,
                                  **batch_throughput(ctx, models))), flush=True)
        elif which == "sweep":
            # f3: speed-up against reduction factor on the two synthetic stand-ins, plain and learned
            n = int(argv[2]) if len(argv) > 2 else 200_000
            out_path = argv[3] if len(argv) > 3 else None
            cases = [("AMR (clump octree)",
                      lambda s_, n_: synth.octree_model(n_, seed=s_, n_lines=1, n_freq=50, l_min=2, l_max=2),
                      (0.90, 2.10, 0.10), 3),
                     ("SPH (binary-wind spiral)", lambda s_, n_: synth.spiral_model(n_, seed=s_, n_freq=50),
                      (1.00, 2.15, 0.21), 4)]
            from . import learned
            allres = []
            for name, mk, t1, test_seed in cases:
                Xs, ys = [], []
                for s_ in (100, 101):
                    mt = mk(s_, n // 2)
                    X, y = learned.training_samples(ctx, mt, [(t1[0] * k, t1[1] * k, t1[2], 1000 + 10 * s_ + j)
                                                              for j, k in enumerate((1.0, 1.5, 2.2))])
                    Xs.append(X)
                    ys.append(y)
                std, _, _ = learned.train_network(ctx, np.concatenate(Xs), np.concatenate(ys), epochs=40, seed=1)
                res = reduction_sweep(ctx, mk(test_seed, n), t1, scales=(1.0, 1.3, 1.7, 2.2, 3.0), std=std)
                res.update(experiment="reduction_sweep", model=name, table1=t1)
                allres.append(res)
                print(json.dumps({k: v for k, v in res.items() if k != "runs"} | {"runs": [
                    {k: v for k, v in r.items() if not k.startswith("cdf")} for r in res["runs"]]}), flush=True)
            if out_path:
                with open(out_path, "w") as f:
                    json.dump(allres, f)
        elif which == "learned4":
            # the binary-wind spiral: training seeds 100-103 at n_train points, the
            # test seed 4 at n_test particles (1 line x 100 bins, l = 2)
            n_test = int(argv[2]) if len(argv) > 2 else 1_000_000
            n_train = int(argv[3]) if len(argv) > 3 else 150_000
            t0 = time.perf_counter()
            test = synth.spiral_model(n_test, seed=4)
            gen = time.perf_counter() - t0
            res = learned_reduction_study(ctx, lambda s_: synth.spiral_model(n_train, seed=s_),
                                          (100, 101, 102, 103), test, (1.00, 2.15, 0.21))
            print(json.dumps(dict(experiment="learned_reduction_study", model="SPH (binary-wind spiral)",
                                  n_train=n_train, generation_s=gen, **res)), flush=True)
        elif which == "learned":
            n = int(argv[2]) if len(argv) > 2 else 20000

            def octree(s_):
                return synth.octree_model(n, seed=s_, hi_level=7, n_lines=1, n_freq=20, l_min=1, l_max=1)

            def spiral(s_):
                return synth.spiral_model(n, seed=s_, n_freq=20, level=1)

            for name, mk, t1, test_seed in (("AMR (clump octree)", octree, (0.90, 2.10, 0.10), 3),
                                            ("SPH (binary-wind spiral)", spiral, (1.00, 2.15, 0.21), 4)):
                for frac in ((0.2, 0.1) if len(argv) <= 3 else tuple(float(x) for x in argv[3].split(","))):
                    print(json.dumps(dict(experiment="learned_vs_plain", model=name, table1=t1,
                                          **learned_vs_plain(ctx, mk, (100, 101, 102, 103), test_seed, t1,
                                                             keep_fraction=frac))), flush=True)
        else:
            n = int(argv[2]) if len(argv) > 2 else 200000
            cases = [("AMR (clump octree)", synth.octree_model(n, seed=3, n_lines=1, n_freq=50, l_min=2, l_max=2),
                      (0.90, 2.10, 0.10)),
                     ("SPH (binary-wind spiral)", synth.spiral_model(n, seed=4, n_freq=50), (1.00, 2.15, 0.21))]
            for name, m, prm in cases:
                print(json.dumps(dict(experiment="reduction_speedup", model=name, table1=prm,
                                      **reduction_speedup(ctx, m, *prm))), flush=True)
    finally:
        ctx.close()


if __name__ == "__main__":
    main(sys.argv)
