"""The allocation-free primal residual entry point against the solver's own.

scylla_primal_residual_noalloc serves callers that cannot allocate device memory
(plugins handed a fixed memory pool, loops that forbid allocator calls): it keeps its
reduction scratch in a fixed device array.  Its eps_p must equal the one scylla_pdhg_solve
reports for the same point (a zero-iteration solve evaluates the current point),
within the tolerance of the parity tests, on two calls in a row (the second call
reuses the scratch the first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = 1e-9


def test_noalloc_residual_matches_solver_twice():
    import torch

    S = lib()
    inst = I.packing_covering(m=3000, n=6000, per_col=8, seed=77)
    lp = S.LP.from_instance(inst, S.default_params(aux_general_integers=0))
    _, _, eta, omega = lp.get_state()
    dev = torch.device("cuda")
    rowptr = torch.tensor(inst.rowptr, dtype=torch.int64, device=dev)
    cols = torch.tensor(inst.cols, dtype=torch.int32, device=dev)
    vals = torch.tensor(inst.vals, dtype=torch.float64, device=dev)
    lo = torch.tensor(inst.lo, dtype=torch.float64, device=dev)
    hi = torch.tensor(inst.hi, dtype=torch.float64, device=dev)
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(5)
    for trial in range(2):
        x = rng.uniform(inst.l, inst.u) * (0.5 + trial)
        x = np.minimum(x, inst.u)
        lp.set_state(x, np.zeros(inst.m), eta, omega)
        r = lp.pdhg_solve(0.0, 0)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        S.primal_residual_noalloc(inst.m, rowptr.data_ptr(), cols.data_ptr(), vals.data_ptr(), xd.data_ptr(),
                                  lo.data_ptr(), hi.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        rn, eps_p = out.cpu().numpy()
        assert abs(eps_p - r.eps_p) <= TOL * max(1.0, r.eps_p), (trial, eps_p, r.eps_p)
        ax = inst.csr() @ x
        ref = float(np.linalg.norm(ax - np.clip(ax, inst.lo, inst.hi)))
        assert abs(rn - ref) <= TOL * max(1.0, ref), (trial, rn, ref)
    lp.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    S = lib()
    with pytest.raises(S.ScyllaError) as ei:
        S.primal_residual_noalloc(2_097_153, 1, 1, 1, 1, 1, 1, 1)
    assert ei.value.code == S.ERR_INVALID_ARG and "2097152" in str(ei.value)
