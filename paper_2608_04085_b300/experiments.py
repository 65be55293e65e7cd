"""The paper's forward comparison runs (Sec. 3.5, Tab. comp_runs; Sec. 4.3
and App. B), composed from the library's entry points: for one configuration,
the CNOP seed, the random seed it started from, the five-mode seed and the
90%-power seed advance in one batch, each with its KE(t) and h_mix(t) series
and its objective at the horizon. Marshalling only: every number comes from
librt_cnop.so."""
from __future__ import annotations

import numpy as np

from . import (RT_FP64, RT_RECON_2D_POWER, RT_RECON_X_MODES, Context)

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
