"""Autotuner for the batched PageRank schedule.

The tile shape is fixed (32 rows, one per lane; the gather step was chosen
by a build-time sweep on the single large space); what varies with the
workload is the schedule of a batch: which jobs get dedicated blocks
(`split`), how many (`grain`), how large the grid is (`max_blocks`) and how
wide its blocks are (`block_warps`: 8 warps, several blocks per SM; 16, one
block per SM with room for every job pointer in registers; or 24, one block
per SM), the order (`claim`): fixed per-block lists, blocks claiming
jobs as they free up, or the sweep, where every job advances one step per
phase on the whole grid, and the least work per warp of a group
(`min_tiles`: more blocks share a job's rows, which keeps each block's
gathers closer together in its L1, but every block of the group pays the
per-iteration barrier).  ``tune`` runs the batch once per candidate (same
workspace, re-planned), times it with CUDA events and leaves the fastest
plan in place.

The plan balances the blocks with a cost model per job (edges + 20 x nodes,
times an iteration estimate); what a job really costs also depends on how
its edges pack into tile descriptors and on where its FP32 iteration stops.
So ``tune`` also re-plans its fastest candidates with the per-job
block-seconds each of them measured (``pagerank_batch_times``) in place of
the model, and keeps such a plan when it is faster.  Results never depend
on the tuning, only the time does.
"""
from __future__ import annotations

import json
import os

import numpy as np

# (split, grain, max_blocks, block_warps, claim[, fp64_form, min_tiles])
CANDIDATES = (
    (1.0, 1.0, 0, 8, 0),
    (0.5, 0.25, 0, 8, 0),
    (1.0, 1.0, 0, 16, 0),
    (0.5, 0.1, 0, 16, 0),
    (0.1, 0.02, 0, 16, 0),
    (0.05, 0.005, 0, 16, 0),
    (0.02, 0.002, 0, 16, 0),
    (0.5, 0.1, 0, 24, 0),
    (0.1, 0.02, 0, 24, 0),
    (0.05, 0.005, 0, 24, 0),
    (0.02, 0.002, 0, 24, 0, 0, 8),
    (0.05, 0.005, 0, 24, 1, 0, 4),
    (0.02, 0.002, 0, 24, 1, 0, 8),
    (0.01, 0.001, 0, 24, 1, 0, 4),
    (0.05, 0.005, 0, 16, 1),
    (1.0, 1.0, 0, 24, 2),
    (1.0, 1.0, 0, 16, 2),
)
MEASURED = 3  # candidates re-planned with measured job costs


def _time(batch, reps):
    import torch
    batch.run()
    batch.query()                      # warm-up run of this plan
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run()
        e1.record()
        batch.query()
        ms.append(e0.elapsed_time(e1))
    return min(ms)


def tune(batch, candidates=CANDIDATES, reps: int = 1, table_path: str | None = None,
         measured: int = MEASURED):
    """Pick the fastest schedule for ``batch`` (a PageRankBatch); returns
    (best candidate tuple, {candidate: ms}).
    Candidates re-planned with measured job costs are keyed with a
    ``+measured`` suffix; the chosen plan's costs stay in ``batch.job_cost``."""
    times, costs = {}, {}
    for cand in candidates:
        batch.replan(cand)
        times[(cand, False)] = _time(batch, reps)
        costs[cand] = np.maximum(batch.times(), 1e-9)  # a cost must be positive
    # job costs only place jobs on blocks: the sweep order has no placement
    placed = [c for c in candidates if len(c) < 5 or c[4] != 2]
    for cand in sorted(placed, key=lambda c: times[(c, False)])[:measured]:
        batch.replan(cand, job_cost=costs[cand])
        times[(cand, True)] = _time(batch, reps)
    best_key = min(times, key=times.get)
    best, use_cost = best_key
    batch.replan(best, job_cost=costs[best] if use_cost else None)
    if table_path:
        key = f"jobs={batch.plan.n_jobs},graphs={batch.plan.n_graphs}," \
              f"edges={sum(g.n_edges for g in batch.graphs)},prec={batch.prec}"
        table = {}
        if os.path.exists(table_path):
            with open(table_path) as fh:
                table = json.load(fh)
        table[key] = {"split": best[0], "grain": best[1], "max_blocks": best[2],
                      "block_warps": best[3], "claim": best[4],
                      "min_tiles": best[6] if len(best) > 6 else 0,
                      "measured_costs": use_cost, "ms": times[best_key]}
        with open(table_path, "w") as fh:
            json.dump(table, fh, indent=1)
    return best, {"/".join(map(str, c)) + ("+measured" if m else ""): round(t, 3)
                  for (c, m), t in times.items()}
