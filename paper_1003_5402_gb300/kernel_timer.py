"""Time one kernel class of the column-generation path on a synthetic workload.

    python -m paper_1003_5402_gb300.kernel_timer --workload prostate --apertures 50 \
        --kernel master_pass --pool 50 --reps 3

Builds the plan of ``--apertures`` apertures with host-driven launches (so that
the number of launches of each class before the timing is known and printed),
then times ``--reps`` launches of ``--kernel`` at pool size ``--pool`` with
dao_k_time (the launches captured into one CUDA graph, one warm replay, one
timed replay).  The printed ``launches_before`` of the kernel class plus
``--reps`` (the warm replay) is the number of launches of that kernel to skip
when a profiler should see exactly the timed launches.  ``--kernel
master_solve`` reports the plan's own persistent master launches (one per
pool size 1 .. apertures) and the evaluations of each.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="prostate")
    ap.add_argument("--apertures", type=int, default=50)
    ap.add_argument("--kernel", default="master_pass")
    ap.add_argument("--pool", type=int, default=0, help="pool size K for the master kernels (default: --apertures)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp16", "bf16"))
    a = ap.parse_args(argv)

    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import phantom as P
    from . import binding
    from .binding import Plan

    case = P.make_case(P.CONFIGS[a.workload]())
    prec = {"fp32": binding.DAO_PREC_FP32, "fp16": binding.DAO_PREC_FP16, "bf16": binding.DAO_PREC_BF16}[a.precision]
    stream = torch.cuda.Stream()
    with Plan(case, stream=stream.cuda_stream, precision=prec) as plan:
        plan.profile_enable(True)
        plan.solve(a.apertures)
        before = {kc: plan.profile_read(kc) for kc in binding.KC if kc != "other"}
        plan.profile_enable(False)
        evals = [int(e) for e in plan.master_stats()[0]]
        K = a.pool or a.apertures
        out = {"workload": a.workload, "kernel": a.kernel, "pool": K, "reps": a.reps, "voxels": case.n_voxels,
               "nnz": case.nnz, "precision": a.precision, "evaluations_per_solve": evals}
        if a.kernel == "master_solve":
            # the persistent solve cannot be re-run in place: report the plan's own launches
            n, ms = before["master_solve"]
            out.update(us_per_launch=round(1e3 * ms / max(n, 1), 3), launches=n)
        else:
            out.update(us_per_launch=round(plan.k_time(a.kernel, K, a.reps), 3),
                       launches_before=before[a.kernel][0])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
