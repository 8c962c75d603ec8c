"""Write ``oracle/op_counts.json``: the method's floating-point operations
per unit of each step, measured by the oracle's counting build.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: it runs the oracle
(the plain build to advance the state, the counting build ``op_count.cpp``
to count) and writes a data file that ``bench.py`` reads to state a
kernel's achieved rate in the method's own operations (the roofline
numerator).

Counted: one SSP-RK3 step of the benchmark's workload (the ``sweep_box``
recipe at 256^3, FP64) after `warm` steps of the plain oracle, as the
benchmark times steps after its warm-up; each distinct operation counted
once per unit (``cse``: the oracle's recomputation of shared subexpressions
removed), every 16th unit of each step sampled.  Units: c2p and assemble
per cell, faces per face, emf per edge, ct (the face-field update) per
face, rk per updated value.  The inversion's count is also split into a
part per cell and a part per Newton iteration, from a second counted step
taken from the initial state (whose exact Newton memory needs fewer
iterations): a + b * iterations.

    python -m oracle.count_ops [n] [warm] [sample_every]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "op_counts.json")


def main(n: int = 256, warm: int = 3, sample_every: int = 16) -> dict:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as orc
    from paper_1810_04597_gb300 import inputs
    prob = inputs.sweep_box(n)
    cfg = orc.make_cfg(prob)
    t0 = time.time()
    st0, Z0 = orc.p2c(cfg, prob.prims, prob.bface)
    cold, cold_stats = orc.count_steps(cfg, None, None, 1, sample_every=sample_every, cse=True, state=st0, Z=Z0)
    stw, Zw, _, _ = orc.steps(cfg, st0, Z0, warm)
    counts, stats = orc.count_steps(cfg, None, None, 1, sample_every=sample_every, cse=True, state=stw, Z=Zw)
    per_unit = {k: v["per_unit"] for k, v in counts.items() if v["per_unit"]}
    its = stats["iters"] / stats["calls"]
    its0 = cold_stats["iters"] / cold_stats["calls"]
    c2p_w, c2p_0 = counts["c2p"]["per_unit"], cold["c2p"]["per_unit"]
    per_it = (c2p_w - c2p_0) / (its - its0)
    out = {
        "workload": f"sweep_box {n}^3, one SSP-RK3 step after {warm} steps of the plain oracle, FP64",
        "rule": "operations +, -, *, / and sqrt, each 1; each distinct operation (kind and operand values) "
                "counted once per unit; no operation with an exact 0 or +-1 operand that makes it trivial; "
                "metric evaluation, coordinates and selections (min, max, minmod) not counted",
        "sample_every": sample_every,
        "flops_per_unit": per_unit,
        "units": {k: v["units"] for k, v in counts.items() if v["units"]},
        "ops_per_unit": {k: {op: v[op] / v["sampled"] for op in ("add", "mul", "div", "sqrt")}
                         for k, v in counts.items() if v["sampled"]},
        "c2p_newton_iters_per_cell": its,
        "c2p_per_cell_fixed": c2p_w - per_it * its,
        "c2p_per_newton_iteration": per_it,
        "from_initial_state": {"flops_per_unit": {k: v["per_unit"] for k, v in cold.items() if v["per_unit"]},
                               "c2p_newton_iters_per_cell": its0},
        "update_per_cell": per_unit.get("assemble", 0.0) + 3.0 * per_unit.get("ct", 0.0)
                           + 8.0 * per_unit.get("rk", 0.0),
        "seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    return out


if __name__ == "__main__":
    args = [int(a) for a in sys.argv[1:]]
    print(json.dumps(main(*args), indent=1, sort_keys=True))
