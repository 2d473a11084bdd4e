"""Per-iteration log of a reconstruction, one JSON object per line.

The solve runs one ADMM iteration at a time through the checkpoint path of
``selr_solve`` (``state_inout`` / ``resume``), which continues bit for bit, so
the logged run ends with exactly the X of an uninterrupted run of the same
length.  After each iteration one line records:

* ``iteration``: k (1-based);
* ``rel_change``: ||X^k - X^(k-1)||^2 / ||X^(k-1)||^2, the stopping quantity of
  Algorithms S1 / S2 (for a parameter model the largest over the FE positions);
* ``rank_hist``: for each lift family, {number of singular values above the
  threshold: number of matrices} of this iteration's SVTs (eigensolver
  families; families solved by the warp-per-matrix Jacobi SVT report none);
* ``mean_rank``: the mean of those counts per family;
* ``ms``: the iteration's device time (CUDA events on the solve stream);
* ``status``: the plan's status word after the iteration (0 = clean).
"""
from __future__ import annotations

import json

import torch

from . import api


def _families(plan):
    two_d = plan.desc.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV")
    return ("row", "col") if two_d else ("pe", "param")


def run_logged(plan, Y, mask, X_out, n_iter, out, stream=None):
    """Run ``n_iter`` iterations of ``plan`` on (Y, mask) into X_out, writing one
    JSON line per iteration to ``out`` (a path or a text file object).  Returns
    the list of records."""
    if n_iter < 1:
        raise ValueError("n_iter must be >= 1")
    stream = stream if stream is not None else torch.cuda.current_stream()
    state = api.new_state(plan, device=Y.device)
    plan.set_iterations(1)
    fams = _families(plan)
    sizes = [plan.lift_shape(a)[0] for a in fams]
    records = []
    own = isinstance(out, str)
    f = open(out, "w") if own else out
    try:
        for k in range(n_iter):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                _, rel = api.selr_solve(plan, Y, mask, X_out, state=state, resume=k > 0, stream=stream)
            e1.record(stream)
            e1.synchronize()
            st = api.selr_sync_status(plan, stream)
            sums, its = api.selr_plan_rank_sums(plan, stream)
            hist, mean = {}, {}
            o = 0
            for name, nm in zip(fams, sizes):
                r = sums[o:o + nm] // max(its, 1)
                o += nm
                if r.any():
                    vals, cnt = torch.unique(torch.from_numpy(r), return_counts=True)
                    hist[name] = {int(v): int(c) for v, c in zip(vals.tolist(), cnt.tolist())}
                    mean[name] = float(r.mean())
            rec = {"iteration": k + 1, "rel_change": float(rel), "rank_hist": hist, "mean_rank": mean,
                   "ms": float(e0.elapsed_time(e1)), "status": int(st)}
            records.append(rec)
            f.write(json.dumps(rec) + "\n")
            f.flush()
    finally:
        if own:
            f.close()
    return records
