"""Write reference_objectives.json: optimal objectives of seeded LP relaxations,
computed by the FP64 CPU oracle alone (PDHG to relative KKT error <= 1e-8).

These are the FP64-oracle values against which the objective error of the GPU
solves (FP64 and FP32-mixed) is stated.  Usage:
    python tests/golden/make_reference_objectives.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pdhg as O  # noqa: E402
from paper_2307_03466_gb300 import instances as I  # noqa: E402

WORKLOADS = {
    "packcover_m50k_n100k_nnz1M": lambda: I.packing_covering(m=50_000, n=100_000, per_col=10, seed=1002),
}


def main():
    out = {"citation": "objectives of the LP relaxation (Algorithm 1 input, relaxed) from oracle.pdhg "
                       "solved to relative KKT error <= 1e-8 (Section 2.2 stopping rule)", "workloads": {}}
    for name, make in WORKLOADS.items():
        inst = make()
        lp = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        t0 = time.time()
        r = lp.solve(1e-8, 2_000_000)
        out["workloads"][name] = {"pobj": r.pobj, "dobj": r.dobj, "rel_kkt": r.rel_kkt, "status": r.status,
                                  "iterations": r.iterations, "seconds": time.time() - t0}
        print(name, out["workloads"][name], flush=True)
    json.dump(out, open(os.path.join(HERE, "reference_objectives.json"), "w"), indent=1)


if __name__ == "__main__":
    main()
