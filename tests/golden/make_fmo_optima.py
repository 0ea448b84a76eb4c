"""Writes fmo_optima.txt: the FP64 oracle's beamlet-level FMO optimum
(oracle.fmo: projected Newton with exact factorisations, pinned against
L-BFGS-B in tests/test_oracle_pins.py) of the seeded full-size workloads, which
take the oracle minutes.  Calls only the oracle and the input generator.

    python tests/golden/make_fmo_optima.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import phantom  # noqa: E402

WORKLOADS = ["prostate"]

if __name__ == "__main__":
    lines = ["# workload  F_fmo (oracle.fmo, FP64)  newton_iterations  status"]
    for name in WORKLOADS:
        r = oracle.fmo(phantom.make_case(phantom.CONFIGS[name]()))
        lines.append(f"{name} {r.F!r} {r.iters} {r.status}")
    with open(os.path.join(HERE, "fmo_optima.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
