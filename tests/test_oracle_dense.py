"""Pins for the oracle's interpolative decomposition (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dense


@pytest.mark.parametrize("m,n,seed", [(40, 9, 0), (12, 30, 1), (64, 64, 2), (7, 7, 3)])
def test_cpqr_matches_lapack_geqp3(m, n, seed):
    """Tie-free Gaussian input: same pivots and |diag R| as LAPACK xGEQP3."""
    M = np.random.default_rng(seed).standard_normal((m, n))
    k, perm, R = dense.cpqr(M, 0.0)
    Q2, R2, P2 = sla.qr(M, pivoting=True, mode="economic")
    assert k == min(m, n)
    np.testing.assert_array_equal(perm[:k], P2[:k])
    np.testing.assert_allclose(np.abs(np.diag(R[:, :k])), np.abs(np.diag(R2)[:k]), rtol=1e-10)


def _decaying(m, n, seed, rate=0.3):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((m, m)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    s = rate ** np.arange(min(m, n))
    return (U[:, :s.size] * s) @ V[:, :s.size].T


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-8])
def test_id_error_bound(tol):
    M = _decaying(60, 25, 4)
    k, perm, T = dense.interp_decomp(M, tol)
    sk, rd = perm[:k], perm[k:]
    _, _, R = dense.cpqr(M, tol)
    err = np.linalg.norm(M[:, rd] - M[:, sk] @ T, 2)
    r11 = abs(R[0, 0])
    assert err <= 10 * tol * r11 * np.sqrt(M.shape[1])
    # rank rule: |R_kk| > tol |R_11| for the kept pivots, next one would fail
    d = np.abs(np.diag(R[:, :k]))
    assert np.all(d > tol * r11)
    assert k < 25


def test_exact_low_rank_reproduced():
    g = np.random.default_rng(5)
    M = g.standard_normal((30, 4)) @ g.standard_normal((4, 12))
    k, perm, T = dense.interp_decomp(M, 1e-12)
    assert k == 4
    np.testing.assert_allclose(M[:, perm[k:]], M[:, perm[:k]] @ T, atol=1e-11 * np.abs(M).max())


def test_special_ranks():
    assert dense.interp_decomp(np.zeros((5, 3)), 1e-3)[0] == 0
    M = np.random.default_rng(6).standard_normal((8, 5))
    assert dense.interp_decomp(M, 0.0)[0] == 5
    # more columns than rows: rank at most m
    M = np.random.default_rng(7).standard_normal((3, 6))
    assert dense.interp_decomp(M, 0.0)[0] == 3


def test_tie_rule_prefers_lowest_original_index():
    g = np.random.default_rng(8)
    c = g.standard_normal(10)
    M = np.column_stack([0.5 * c, g.standard_normal(10) * 0.1, c, -c])  # cols 2 and 3 tie
    log = []
    k, perm, R = dense.cpqr(M, 0.0, log)
    assert perm[0] == 2
    assert log and log[0][0] == 0 and log[0][2] == 2
