"""Pins of the oracle's diagonal preconditioning (Section 2.1 hands it to PDLP: Ruiz
equilibration, then Pock-Chambolle with alpha = 1) against closed forms and a
theorem, none of which re-types the oracle's own loop.

* A positive rank-one matrix a_ij = u_i v_j stays rank one under a Ruiz pass that
  takes both norms from the same matrix: after k passes
      a~_ij = (u_i / max u)^(1/2^k) (v_j / max v)^(1/2^k).
  A pass that scaled the rows first and took the column norms afterwards, a
  missing square root, or swapped row and column norms each miss this.
* Pock-Chambolle on a rank-one matrix p_i q_j gives sqrt(p_i q_j) / sqrt(sum p sum q).
* Pock-Chambolle's output has spectral norm at most 1, by the Schur test with
  weights sqrt(row sums) and sqrt(column sums).  Row and column sums exchanged
  violate it on rectangular matrices.
* A permuted diagonal matrix becomes a signed permutation matrix in one Ruiz pass,
  and stays one under Pock-Chambolle.
* Zero rows and columns keep multiplier 1.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.pdhg import precondition


def scaled(A, R, C):
    return (sp.diags(R) @ A @ sp.diags(C)).toarray()


@pytest.mark.parametrize("k", [1, 2, 3, 5, 10])
def test_ruiz_on_positive_rank_one_matches_closed_form(k):
    rng = np.random.default_rng(k)
    u = rng.uniform(0.01, 50.0, 7)
    v = rng.uniform(0.001, 9.0, 11)
    A = sp.csr_matrix(np.outer(u, v))
    R, C = precondition(A, ruiz_iters=k, pock_chambolle=False)
    e = 0.5 ** k
    want = np.outer((u / u.max()) ** e, (v / v.max()) ** e)
    np.testing.assert_allclose(scaled(A, R, C), want, rtol=1e-12, atol=0)


def test_ruiz_then_pock_chambolle_on_rank_one_matches_closed_form():
    rng = np.random.default_rng(5)
    u = rng.uniform(0.1, 30.0, 6)
    v = rng.uniform(0.1, 4.0, 9)
    A = sp.csr_matrix(np.outer(u, v))
    k = 4
    R, C = precondition(A, ruiz_iters=k, pock_chambolle=True)
    p = (u / u.max()) ** (0.5 ** k)
    q = (v / v.max()) ** (0.5 ** k)
    want = np.sqrt(np.outer(p, q)) / np.sqrt(p.sum() * q.sum())
    np.testing.assert_allclose(scaled(A, R, C), want, rtol=1e-12, atol=0)
    # a rank-one matrix with these factors has spectral norm exactly 1
    assert abs(np.linalg.norm(want, 2) - 1.0) < 1e-12


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("ruiz", [0, 10])
def test_pock_chambolle_output_has_spectral_norm_at_most_one(seed, ruiz):
    rng = np.random.default_rng(seed)
    m, n = (30, 70) if seed % 2 else (80, 25)
    A = sp.random(m, n, density=0.15, random_state=seed, data_rvs=lambda s: rng.lognormal(0, 2, s)).tocsr()
    A.data *= rng.choice([-1.0, 1.0], A.nnz)
    R, C = precondition(A, ruiz_iters=ruiz, pock_chambolle=True)
    S = scaled(A, R, C)
    assert np.all(np.isfinite(S))
    assert np.linalg.norm(S, 2) <= 1.0 + 1e-12


def test_permuted_diagonal_becomes_signed_permutation():
    rng = np.random.default_rng(3)
    n = 12
    perm = rng.permutation(n)
    d = rng.uniform(1e-3, 1e3, n) * rng.choice([-1.0, 1.0], n)
    A = sp.csr_matrix((d, (np.arange(n), perm)), shape=(n, n))
    for pc in (False, True):
        R, C = precondition(A, ruiz_iters=1, pock_chambolle=pc)
        S = scaled(A, R, C)
        np.testing.assert_allclose(np.abs(S[np.arange(n), perm]), 1.0, rtol=1e-14)
        assert np.array_equal(np.sign(S[np.arange(n), perm]), np.sign(d))
        assert np.count_nonzero(S) == n


def test_zero_rows_and_columns_keep_unit_multipliers():
    A = sp.csr_matrix(np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 8.0], [0.0, 0.0, 0.0]]))
    R, C = precondition(A, ruiz_iters=10, pock_chambolle=True)
    assert R[0] == 1.0 and R[2] == 1.0 and C[1] == 1.0
    assert np.all(R > 0) and np.all(C > 0)


def _planted(mistake):
    """The preconditioning with one plausible mistake planted."""
    def pre(A, ruiz_iters, pock_chambolle):
        m, n = A.shape
        R, C = np.ones(m), np.ones(n)
        absA = abs(A).tocsr()
        root = (lambda x: x) if mistake == "no_sqrt" else np.sqrt
        for _ in range(ruiz_iters):
            S = sp.diags(R) @ absA @ sp.diags(C)
            rmax = np.asarray(S.max(axis=1).todense()).ravel()
            R = R / root(np.where(rmax > 0, rmax, 1.0))
            if mistake == "rows_first":
                S = sp.diags(R) @ absA @ sp.diags(C)
            cmax = np.asarray(S.max(axis=0).todense()).ravel()
            C = C / root(np.where(cmax > 0, cmax, 1.0))
        if pock_chambolle:
            S = sp.diags(R) @ absA @ sp.diags(C)
            rsum = np.asarray(S.sum(axis=1)).ravel()
            csum = np.asarray(S.sum(axis=0)).ravel()
            if mistake == "sums_exchanged":
                rsum, csum = np.resize(csum, m), np.resize(rsum, n)
            R = R / np.sqrt(np.where(rsum > 0, rsum, 1.0))
            C = C / np.sqrt(np.where(csum > 0, csum, 1.0))
        return R, C
    return pre


@pytest.mark.parametrize("mistake", ["rows_first", "no_sqrt", "sums_exchanged"])
def test_pins_reject_planted_mistakes(monkeypatch, mistake):
    """Each planted mistake fails at least one of the pins above."""
    import sys
    mod = sys.modules[__name__]
    monkeypatch.setattr(mod, "precondition", _planted(mistake))
    pins = [lambda: test_ruiz_on_positive_rank_one_matches_closed_form(3),
            test_ruiz_then_pock_chambolle_on_rank_one_matches_closed_form,
            lambda: test_pock_chambolle_output_has_spectral_norm_at_most_one(1, 0),
            lambda: test_pock_chambolle_output_has_spectral_norm_at_most_one(0, 10),
            test_permuted_diagonal_becomes_signed_permutation]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1
