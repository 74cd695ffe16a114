"""Shared helpers of the GPU parity tests: build the library once, create matching
GPU and oracle LPs from the same seeded instance, and compare iterates."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I

torch = pytest.importorskip("torch")

INF = np.inf


def gpu_available() -> bool:
    return bool(torch.cuda.is_available())


def lib():
    from paper_2307_03466_gb300 import build as B
    from paper_2307_03466_gb300 import scylla as S
    B.build()
    S.lib()
    return S


PDHG_KEYS = ("n_check", "ruiz_iters", "pock_chambolle", "adaptive_step", "restarts", "primal_weight_update",
             "fixed_step_factor", "stall_checks")


def pair(inst, precision=0, **kw):
    """GPU handle and oracle LP of the same instance with the same PDHG parameters
    (no auxiliary columns: the LP relaxation exactly as given)."""
    S = lib()
    gp = S.default_params(precision=precision, aux_general_integers=0)
    op = O.PdhgParams()
    for k, v in kw.items():
        setattr(gp, k, int(v) if k != "fixed_step_factor" else float(v))
        if k in PDHG_KEYS:
            setattr(op, k, v)
    g = S.LP.from_instance(inst, gp)
    int_cols = np.nonzero(inst.is_int)[0]
    o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, int_cols=int_cols, params=op)
    return g, o


def rel_err(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def long_row_instance(seed=7, m=320, n=700):
    """Random LP with a few rows and columns longer than one warp tile (256 nnz) and
    empty rows, to cover the long-row path and ragged tiles."""
    rng = np.random.default_rng(seed)
    dense = np.where(rng.random((m, n)) < 0.01, rng.lognormal(size=(m, n)), 0.0)
    dense[3, :] = rng.uniform(0.5, 2.0, size=n)        # 700-nonzero rows
    dense[100, :] = rng.uniform(0.5, 2.0, size=n)
    dense[:, 11] = rng.uniform(0.5, 2.0, size=m)       # 320-nonzero columns
    dense[:, 500] = rng.uniform(0.5, 2.0, size=m)
    dense[7, :] = 0.0                                  # empty rows
    dense[250, :] = 0.0
    x0 = rng.uniform(1, 9, size=n)
    r = dense @ x0
    s = rng.uniform(0.05, 0.5, size=m)
    cov = rng.random(m) < 0.5
    lo = np.where(cov, r * (1 - s), -INF)
    hi = np.where(cov, INF, r * (1 + s))
    lo[7] = -1.0
    hi[250] = 1.0
    A = sp.csr_matrix(dense)
    A.sort_indices()
    c = rng.normal(size=n)
    return I.Instance("long_rows", m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                      A.data.astype(np.float64), c, lo, hi, np.zeros(n), np.full(n, 10.0),
                      (rng.random(n) < 0.3).astype(np.uint8))


def parity_instances():
    return {
        "setcover_200x500": I.set_cover(),
        "packcover_2kx4k": I.packing_covering(m=2000, n=4000, per_col=10, seed=11),
        "long_rows": long_row_instance(),
        "mcf_small": I.mcf(nodes=30, avg_degree=4, commodities=12, seed=5),
        "knapcover_700": I.knapsack_cover(700, seed=3),
    }
