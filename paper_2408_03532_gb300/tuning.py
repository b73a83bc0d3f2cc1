"""Time to a target error for Algorithm 3, and the step-size search behind it.

Section 4 tunes the PFT phase's step size and its TV weight on a logarithmic
grid before timing the hybrid against plain PIE. This module does the same on
the GPU, entirely through the library's warm_start_then_refine (Algorithm 3):

* sweeps_to_target: a traced run (per-sweep phase-aligned NRMSE against a
  known object) gives the number of refine-phase sweeps a schedule needs to
  reach a target error;
* time_to_target: that run, then the same schedule with exactly that many
  full sweeps and no error tracing, timed as wall time around the call (the
  call synchronises once per sweep for its stopping rule, as a user's call
  does);
* search: every schedule of a grid ranked by its modelled time (measured wall
  time per sweep of each kind times the sweeps it needs).

Every run starts from a copy of the same start in one device buffer, so the
library's captured sweep graphs are reused from run to run.
"""
from __future__ import annotations

import itertools
import statistics
import time
from dataclasses import replace

from . import pft


def _run(ctx, buf, z0, schedule, truth=None):
    buf.copy_(z0)
    return ctx.warm_start_then_refine(buf, schedule, truth)


def _wall(ctx, buf, z0, schedule, reps):
    import torch
    ts = []
    for _ in range(reps):
        buf.copy_(z0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.warm_start_then_refine(buf, schedule)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    return statistics.median(ts)


def sweep_costs(ctx, buf, z0, tv: float = 0.0, sweeps: int = 8, reps: int = 3) -> dict:
    """Wall seconds per sweep through warm_start_then_refine: a full sweep, a
    coloured and a batched PFT sweep, and a coloured PFT sweep followed by a
    TV step of weight `tv` (when tv > 0)."""
    full = pft.Schedule(1.0, 1.0, 0.0, 0.0, 0, sweeps)
    col = pft.Schedule(1.0, 1.0, 0.0, 0.0, sweeps, 0)
    out = {}
    for name, s in (("full", full), ("pft_coloured", col), ("pft_batched", replace(col, pft_batched=True))) + (
            (("pft_coloured_tv", replace(col, tv_pft=tv)), ("pft_batched_tv", replace(col, tv_pft=tv,
                                                                                     pft_batched=True)))
            if tv > 0 else ()):
        _wall(ctx, buf, z0, s, 1)  # captures the sweep graphs
        out[name] = _wall(ctx, buf, z0, s, reps) / sweeps
    return out


def sweeps_to_target(ctx, buf, z0, truth, schedule, target: float):
    """(PFT sweeps run, full sweeps needed or None, traced NRMSE per sweep)."""
    tr = _run(ctx, buf, z0, schedule, truth)
    k = sum(1 for t in tr if t["phase"] == "pft")
    for i, t in enumerate(tr):
        if t["nrmse"] <= target and (t["phase"] == "full" or schedule.max_full == 0):
            return k, (i + 1 - k if t["phase"] == "full" else 0), [t["nrmse"] for t in tr]
    return k, None, [t["nrmse"] for t in tr]


def time_to_target(ctx, buf, z0, truth, schedule, target: float, reps: int = 3) -> dict:
    """Wall time of Algorithm 3 to `target` through warm_start_then_refine."""
    k, nf, trace = sweeps_to_target(ctx, buf, z0, truth, schedule, target)
    out = {"schedule": schedule_dict(schedule), "pft_sweeps": k, "full_sweeps": nf, "reached": nf is not None,
           "nrmse_trace": [round(e, 5) for e in trace], "best_nrmse": min(trace) if trace else None}
    if nf is None:
        out["s"] = None
        return out
    timed = replace(schedule, max_pft=k, tol_pft=0.0, max_full=nf, tol_full=0.0)
    _wall(ctx, buf, z0, timed, 1)
    out["s"] = _wall(ctx, buf, z0, timed, reps)
    return out


def schedule_dict(s) -> dict:
    return {"beta_pft": s.beta_pft, "beta_full": s.beta_full, "tol_pft": s.tol_pft, "max_pft": s.max_pft,
            "tv_pft": s.tv_pft, "tv_full": s.tv_full, "pft_batched": bool(s.pft_batched)}


def search(ctx, buf, z0, truth, target: float, max_full: int, betas, tvs, counts, modes=(False, True),
           costs: dict | None = None) -> list[dict]:
    """Ranks the schedules of the grid betas x tvs x counts x modes (False:
    coloured PFT phase, exact Algorithm 3 order; True: batched PFT phase) by
    modelled wall time to `target`: PFT sweeps x their cost + full sweeps x
    the full sweep's cost (costs from sweep_costs, measured here if not given;
    a TV step costs the same at every weight and is folded into the PFT sweep
    cost). Unreached schedules last."""
    costs = costs or sweep_costs(ctx, buf, z0, tv=1e-2)
    rows = []
    for batched, beta, tv, k in itertools.product(modes, betas, tvs, counts):
        key = ("pft_batched" if batched else "pft_coloured") + ("_tv" if tv > 0 else "")
        s = pft.Schedule(beta, 1.0, 0.0, 0.0, k, max_full, tv_pft=tv, pft_batched=batched)
        kk, nf, trace = sweeps_to_target(ctx, buf, z0, truth, s, target)
        model = None if nf is None else kk * costs[key] + nf * costs["full"]
        rows.append({"pft_batched": batched, "beta_pft": beta, "tv_pft": tv, "pft_sweeps": kk, "full_sweeps": nf,
                     "model_s": model, "pft_end_nrmse": trace[kk - 1] if kk else None})
    rows.sort(key=lambda r: (r["model_s"] is None, r["model_s"] or 0.0))
    return rows
