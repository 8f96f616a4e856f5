"""Coarsest-grid solve of the AMG V-cycle: the explicit inverse of the dense
coarsest operator (Gauss-Jordan with partial pivoting). A one-level
hierarchy (max_levels = 1) makes the V-cycle exactly x = A^{-1} b, checked
against LAPACK's solve of the same matrix: sizes from 1 row to past the
capacity of the thread-block-cluster kernel (whose rows are split over the
cluster's CTAs, ragged at the last one), matrices that need row exchanges,
and a singular matrix, which must come back as a setup error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

thermo = pytest.importorskip("paper_1902_00095_gb300.thermo")


def dense_csr(A):
    n = A.shape[0]
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    return rp, col, np.ascontiguousarray(A, np.float64).ravel()


def one_level_solve(A, b):
    g = thermo.AMG(*dense_csr(A), max_levels=1)
    try:
        n, _ = g.info()
        assert len(n) == 1 and n[0] == A.shape[0]
        return g.vcycle(b)
    finally:
        g.close()


@pytest.mark.parametrize("n", [1, 2, 31, 300, 512, 641, 700])
def test_coarse_inverse_solves_well_conditioned(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    b = rng.standard_normal(n)
    x = one_level_solve(A, b)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [5, 97, 400])
def test_coarse_inverse_pivots(n):
    """Tiny diagonal, large entries elsewhere: elimination without row
    exchanges would divide by ~1e-9; a permutation-like dominant part also
    makes the pivot row differ from the step index at every step."""
    rng = np.random.default_rng(100 + n)
    perm = rng.permutation(n)
    A = 1e-3 * rng.standard_normal((n, n))
    A[np.arange(n), perm] += 1.0 + rng.random(n)
    A[np.arange(n), np.arange(n)] = 1e-9 * (1.0 + rng.random(n))
    b = rng.standard_normal(n)
    x = one_level_solve(A, b)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(ref)


def test_singular_coarsest_is_a_setup_error():
    A = np.ones((40, 40)) + np.diag(np.r_[np.zeros(39), 1.0])
    A[:, 7] = A[:, 3]  # two equal columns: singular, nonzero diagonal
    with pytest.raises(thermo.ThermoError) as e:
        thermo.AMG(*dense_csr(A), max_levels=1)
    assert "singular" in str(e.value)
