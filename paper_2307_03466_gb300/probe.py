"""Short solve of a named workload, for profiler captures.

    python -m paper_2307_03466_gb300.probe <workload> <precision> <attempts> [launch mode]

workload: packcover (m=50k, n=100k, 1M nnz), mcf (n=8.82M, m=1.82M, 25.6M nnz) or
mcf_small (600 nodes, 150 commodities); precision: 0 FP64, 1 FP32-mixed; launch
mode: scylla_params.use_graph (default 1).  Runs `attempts` PDHG attempts from the
cold start (tolerance 0) and prints the attempt count, final relative KKT error,
device seconds and kernel launches.
"""
import sys

from . import build as B
from . import instances as I
from . import scylla as S

WORKLOADS = {
    "packcover": lambda: I.packing_covering(),
    "mcf": lambda: I.mcf(),
    "mcf_small": lambda: I.mcf(nodes=600, avg_degree=8, commodities=150, seed=1003),
}


def main(argv):
    name, prec, attempts = argv[0], int(argv[1]), int(argv[2])
    mode = int(argv[3]) if len(argv) > 3 else 1
    B.build()
    inst = WORKLOADS[name]()
    lp = S.LP.from_instance(inst, S.default_params(precision=prec, aux_general_integers=0, use_graph=mode))
    r = lp.pdhg_solve(0.0, attempts)
    print(name, prec, mode, r.iterations, r.rel_kkt, r.seconds, r.launches)


if __name__ == "__main__":
    main(sys.argv[1:])
