"""The stored transpose A~^T of an LP handle (the matrix the primal step gathers
over), built on the device by a stable radix sort of the nonzeros by column, against
scipy's transpose of the same matrix scaled by the handle's own diagonal scaling, and
against the host-thread construction (scylla_params.host_transpose = 1), bit for bit.
The instances include empty rows and columns, long rows and long columns."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, long_row_instance

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def sparse_edges(seed=3):
    """An LP with empty rows, empty columns and one column in nearly every row."""
    rng = np.random.default_rng(seed)
    m, n = 3000, 5000
    k = 30000
    rows = rng.integers(0, m, k)
    cols = rng.integers(0, n, k)
    keep = (cols != 17) & ~((rows >= 100) & (rows < 200)) & (cols != 4321)
    rows, cols = rows[keep], cols[keep]
    dense = np.array([i for i in range(m) if not 100 <= i < 200])
    rows = np.concatenate([rows, dense])
    cols = np.concatenate([cols, np.full(len(dense), 4321)])
    vals = 1.0 + rng.random(len(rows))
    return I._from_coo("edges", m, n, rows, cols, vals, c=rng.normal(size=n), lo=np.full(m, -1.0), hi=np.full(m, 1.0),
                       l=np.zeros(n), u=np.ones(n), is_int=np.zeros(n, dtype=np.uint8))


INSTANCES = {
    "set_cover": lambda: I.set_cover(),
    "packcover": lambda: I.packing_covering(m=2000, n=4000, per_col=10, seed=11),
    "long_rows": lambda: long_row_instance(),
    "mcf_small": lambda: I.mcf(nodes=30, avg_degree=4, commodities=12, seed=5),
    "edges": sparse_edges,
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(INSTANCES))
def test_device_transpose_matches_scipy_and_host(name, precision):
    S = lib()
    inst = INSTANCES[name]()
    got = []
    for host in (0, 1):
        lp = S.LP.from_instance(inst, S.default_params(precision=precision, aux_general_integers=0, host_transpose=host))
        colptr, rows, vals = lp.transpose()
        R, Cc = lp.scaling()
        got.append((colptr, rows, vals))
        lp.close()
    (cp_d, r_d, v_d), (cp_h, r_h, v_h) = got
    np.testing.assert_array_equal(cp_d, cp_h)
    np.testing.assert_array_equal(r_d, r_h)
    np.testing.assert_array_equal(v_d, v_h)
    A = inst.csr()
    As = (sp.diags(R) @ A @ sp.diags(Cc)).tocsc()
    As.sort_indices()
    np.testing.assert_array_equal(cp_d, As.indptr)
    np.testing.assert_array_equal(r_d, As.indices)
    np.testing.assert_allclose(v_d, As.data, rtol=1e-15, atol=0)


def test_device_transpose_of_the_mcf_workload_matches_scipy():
    """25.6M nonzeros, 8.8M columns (three radix passes)."""
    S = lib()
    inst = I.mcf()
    lp = S.LP.from_instance(inst, S.default_params(precision=1, aux_general_integers=0))
    colptr, rows, _ = lp.transpose()
    lp.close()
    At = inst.csr().tocsc()
    At.sort_indices()
    np.testing.assert_array_equal(colptr, At.indptr)
    np.testing.assert_array_equal(rows, At.indices)
