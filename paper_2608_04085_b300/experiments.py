"""Experiment drivers composed from the library's entry points (marshalling
only: every number comes from librt_cnop.so).

- comparison_runs: the paper's forward comparison runs (Sec. 3.5, Tab.
  comp_runs; Sec. 4.3 and App. B): for one configuration, the CNOP seed, the
  random seed it started from, the five-mode seed and the 90%-power seed
  advance in one batch, each with its KE(t) and h_mix(t) series and its
  objective at the horizon.
- paper_run: one of the paper's three CNOP runs (Tab. runs) from localised
  random starts, followed by comparison_runs for each seed.
- horizon_sweep: CNOPs of one box for several horizons T in one batch, with
  J of the CNOP, the random start and the five-mode seed per T.
- precision_comparison: the CNOP of one box in FP32 state and in FP64 from
  the same start under revolve checkpointing; J errors and the CNOP cosine.
"""
from __future__ import annotations

import numpy as np

from . import (RT_FP32_STATE, RT_FP64, RT_RECON_2D_POWER, RT_RECON_X_MODES, Context)

SEEDS = ("CNOP", "Random", "5modes", "90%Power-2D")


def comparison_runs(problem, v_cnop, v_random, eps, every, precision=RT_FP64, modes=5, power=0.9):
    """Returns {seed name: {"v", "J", "J_ke", "t", "KE", "h_mix"}} for the
    four seeds of one configuration (all scaled to C = eps)."""
    v_cnop = np.asarray(v_cnop, dtype=np.float64).ravel()
    v_random = np.asarray(v_random, dtype=np.float64).ravel()
    with Context([problem], precision=precision) as one:
        rand = one.project(v_random, eps, to_budget=True)
        five, _ = one.reconstruct(v_cnop, RT_RECON_X_MODES, modes, eps)
        p90, _ = one.reconstruct(v_cnop, RT_RECON_2D_POWER, power, eps)
    seeds = [v_cnop, rand, five, p90]
    with Context([problem] * len(seeds), precision=precision) as ctx:
        flat = np.concatenate(seeds)
        J, J_ke, _ = ctx.forward(flat)
        series = ctx.series(flat, every)
    return {name: {"v": seeds[k], "J": J[k], "J_ke": J_ke[k], **series[k]} for k, name in enumerate(SEEDS)}


# The paper's three CNOP runs (Tab. runs): label -> (N, t*, iteration budget).
PAPER_RUNS = {"T2_N128": (128, 2.0, 200), "T2_N256": (256, 2.0, 3000), "T3_N128": (128, 3.0, 5800)}


def paper_run(label, seeds=(0, 1, 2, 3), iters=None, eps=1e-6, h_loc=0.1, precision=RT_FP32_STATE, every=20):
    """One of the paper's CNOP runs on the unit-square configuration (Sec. 2-3,
    Tabs. params and runs), from localised random starts with the given seeds
    (all seeds in one batch): projected L-BFGS to the iteration budget, then
    the comparison seeds of comparison_runs for each. Returns a dict with, per
    seed, the CNOP objective, the kinetic energy at t* of every seed kind, the
    CNOP's KE amplification over its random start and its dominant horizontal
    modes at y_peak."""
    import time
    import rt_inputs
    N, t_star, budget = PAPER_RUNS[label]
    iters = budget if iters is None else iters
    w = rt_inputs.paper_unit_square(N, t_star)
    xi = np.concatenate([rt_inputs.gaussian_field(s, w.ncomp, w.ny, w.nx).ravel() for s in seeds])
    t0 = time.perf_counter()
    with Context([w] * len(seeds), precision=precision) as ctx:
        v0, _, _ = ctx.cnop(xi, eps, 0, h_loc=h_loc)            # the localised random starts
        v, J, res = ctx.cnop(xi, eps, iters, h_loc=h_loc)       # the CNOPs
    solve_s = time.perf_counter() - t0
    n = w.ncomp * w.nx * w.ny
    out = {"label": label, "N": N, "t_star": t_star, "iterations": res["iterations"], "eps": eps,
           "solve_seconds": solve_s, "seeds": []}
    for k, s in enumerate(seeds):
        cmp = comparison_runs(w, v[k * n:(k + 1) * n], v0[k * n:(k + 1) * n], eps, every, precision=precision)
        with Context([w], precision=precision) as one:
            y_peak, E = one.spectrum_x(v[k * n:(k + 1) * n])
        top = [int(m) + 1 for m in np.argsort(-E, kind="stable")[:5]]
        out["seeds"].append({
            "seed": int(s), "J_cnop": float(J[k]), "J_start": float(res["J_history"][0, k]),
            "KE_t_star": {name: float(cmp[name]["J_ke"]) for name in SEEDS},
            "h_mix_t_star": {name: float(cmp[name]["h_mix"][-1]) for name in SEEDS},
            "KE_amplification_vs_random": float(cmp["CNOP"]["J_ke"] / cmp["Random"]["J_ke"]),
            "dominant_modes": top, "y_peak": int(y_peak), "stop": int(res["stop"][k]),
            "chi": float(res["chi"][k])})
    return out


def horizon_sweep(Ts=(1.0, 2.0, 4.0), iters=50, seed=0, eps=1e-4, method=None, precision=RT_FP32_STATE):
    """CNOPs of the 256x768 RT box for several horizons T from one seeded
    i.i.d. (v_x, v_y) start scaled to C = eps, all T in one batch (the
    instances advance in lockstep; each stops at its own horizon), with the
    spectral projected gradient by default; then, per T, J(T) of the CNOP,
    of the random start and of the five-mode seed. Returns a dict."""
    import time
    import rt_inputs
    from . import RT_CNOP_SPG
    method = RT_CNOP_SPG if method is None else method
    ws = [rt_inputs.single_256().replace(T=float(T)) for T in Ts]
    n = ws[0].ncomp * ws[0].nx * ws[0].ny
    xi = np.concatenate([rt_inputs.gaussian_field(seed, ws[0].ncomp, ws[0].ny, ws[0].nx).ravel()] * len(ws))
    t0 = time.perf_counter()
    with Context(ws, precision=precision) as ctx:
        v0, _, _ = ctx.cnop(xi, eps, 0, method=method)          # the random starts
        v, J, res = ctx.cnop(xi, eps, iters, method=method)
    solve_s = time.perf_counter() - t0
    out = {"grid": [ws[0].nx, ws[0].ny], "iterations": res["iterations"], "eps": eps, "method": int(method),
           "solve_seconds": solve_s, "horizons": []}
    for k, w in enumerate(ws):
        vk, v0k = v[k * n:(k + 1) * n], v0[k * n:(k + 1) * n]
        with Context([w], precision=precision) as one:
            five, _ = one.reconstruct(vk, RT_RECON_X_MODES, 5, eps)
        with Context([w] * 3, precision=precision) as three:
            Jc, _, st = three.forward(np.concatenate([vk, v0k, five]))
        out["horizons"].append({"T": float(w.T), "steps": int(st["steps"]), "J_cnop": float(Jc[0]),
                                "J_random": float(Jc[1]), "J_5modes": float(Jc[2]),
                                "J_start": float(res["J_history"][0, k]), "stop": int(res["stop"][k])})
    return out


def precision_comparison(nx=1024, ny=3072, T=6.0, iters=20, seed=0, eps=1e-4, method=None, ckpt_cap_gb=40.0,
                         fp64_cnop=True):
    """CNOP of one RT box in FP32 state and in FP64 from the same seeded
    i.i.d. (v_x, v_y) start (C = eps), revolve checkpointing under a memory
    cap, the projected L-BFGS (the paper's optimiser, Sec. 3.4) by default:
    the relative error of the FP32 J(T) of the FP64 CNOP, the FP32 CNOP's J
    against the FP64 one, and the cosine of the two CNOPs. The cosine
    compares two searches, so it is meaningful once both have converged;
    L-BFGS gets there in far fewer iterations than the spectral projected
    gradient. Defaults: the 1024x3072, T = 6 box.

    fp64_cnop=False runs the FP32 CNOP only and evaluates J of the FP32 CNOP
    and of the start with one FP64 forward each: the FP32 path's error in
    J(T) at those two points, without the FP64 search."""
    import time
    import rt_inputs
    from . import RT_CKPT_REVOLVE, RT_CNOP_LBFGS
    method = RT_CNOP_LBFGS if method is None else method
    w = rt_inputs.rt_box(nx, ny, T=float(T))
    xi = rt_inputs.gaussian_field(seed, w.ncomp, w.ny, w.nx).ravel()
    out = {"grid": [nx, ny], "T": float(T), "iterations": iters, "eps": eps, "runs": {}}
    v = {}
    if not fp64_cnop:
        t0 = time.perf_counter()
        with Context([w], precision=RT_FP32_STATE, ckpt=RT_CKPT_REVOLVE, ckpt_cap_bytes=ckpt_cap_gb * 1e9) as ctx:
            v0, J0, _ = ctx.cnop(xi, eps, 0, method=method)
            v32, J, res = ctx.cnop(xi, eps, iters, method=method)
            _, _, g = ctx.gradient(v32)
            J32_start = float(ctx.forward(v0)[0][0])
        out["runs"]["fp32"] = {"J": float(J[0]), "J_start": float(res["J_history"][0, 0]), "steps": int(g["steps"]),
                               "iterations": int(res["iterations"]), "gradient_evals": int(res["gradient_evals"]),
                               "forward_evals": int(res["forward_evals"]), "seconds": time.perf_counter() - t0,
                               "revolve_recomputed_steps_per_gradient": -int(g["segments"]),
                               "gradient_ms": float(g["ms"])}
        t0 = time.perf_counter()
        with Context([w], precision=RT_FP64) as c64:
            J64_cnop = float(c64.forward(v32)[0][0])
            J64_start = float(c64.forward(v0)[0][0])
        out["fp64_forward_seconds"] = time.perf_counter() - t0
        out["J_fp64_at_fp32_cnop"] = J64_cnop
        out["rel_err_J_fp32_at_fp32_cnop"] = abs(out["runs"]["fp32"]["J"] - J64_cnop) / abs(J64_cnop)
        out["J_fp64_at_start"] = J64_start
        out["rel_err_J_fp32_at_start"] = abs(J32_start - J64_start) / abs(J64_start)
        return out
    for name, prec in (("fp32", RT_FP32_STATE), ("fp64", RT_FP64)):
        t0 = time.perf_counter()
        with Context([w], precision=prec, ckpt=RT_CKPT_REVOLVE, ckpt_cap_bytes=ckpt_cap_gb * 1e9) as ctx:
            v[name], J, res = ctx.cnop(xi, eps, iters, method=method)
            _, _, st = ctx.forward(v[name])
        out["runs"][name] = {"J": float(J[0]), "J_start": float(res["J_history"][0, 0]), "steps": int(st["steps"]),
                             "iterations": int(res["iterations"]), "seconds": time.perf_counter() - t0}
    with Context([w], precision=RT_FP32_STATE) as c32:
        J32_of_v64 = float(c32.forward(v["fp64"])[0][0])
    a, b = v["fp32"], v["fp64"]
    J64 = out["runs"]["fp64"]["J"]
    out["rel_err_J_fp32_at_fp64_cnop"] = abs(J32_of_v64 - J64) / abs(J64)
    out["rel_diff_J_cnop"] = abs(out["runs"]["fp32"]["J"] - J64) / abs(J64)
    out["cnop_cosine"] = float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="the paper's CNOP runs on synthetic random starts")
    ap.add_argument("--run", default="T2_N128", choices=sorted(PAPER_RUNS) + ["horizons", "precision"])
    ap.add_argument("--T", type=float, default=None)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--no-fp64-cnop", action="store_true",
                    help="precision run: FP32 CNOP only, J checked with FP64 forwards")
    a = ap.parse_args()
    if a.run == "horizons":
        print(json.dumps(horizon_sweep(iters=50 if a.iters is None else a.iters)), flush=True)
    elif a.run == "precision":
        print(json.dumps(precision_comparison(T=6.0 if a.T is None else a.T,
                                              iters=20 if a.iters is None else a.iters,
                                              fp64_cnop=not a.no_fp64_cnop)), flush=True)
    else:
        print(json.dumps(paper_run(a.run, seeds=tuple(range(a.seeds)), iters=a.iters)), flush=True)

