"""Dense primitives of Sec. 2: Cholesky and the interpolative decomposition.

The ID (Sec. 2.2, following the cited Cheng-Gimbutas-Martinsson-Rokhlin
construction) is computed by column-pivoted Householder QR of ``A_{R,I}``:
``A_{R,I} P = Q [R11 R12; 0 R22]``, skeletons = the first ``k`` pivot
columns, ``T = R11^{-1} R12`` so that ``A_{R,Ir} ~= A_{R,Is} T``.

Readings where the paper is silent:

* rank: ``k`` = number of leading pivots with ``|R_jj| > tol * |R_11|``
  ("relative precision"); ``R_11 = 0`` gives ``k = 0``; ``tol = 0`` keeps every
  nonzero pivot;
* pivot choice: column norms of the trailing block are recomputed exactly at
  every step (no downdating); the pivot is the candidate with the smallest
  *original* column index among the remaining columns whose squared norm is at
  least ``(1 - 1e-12)`` times the maximum (a deterministic tie rule);
* steps where a second candidate lies within ``1e-10`` relative of the chosen
  one are logged as near-ties.

Parity: pinned against LAPACK xGEQP3 (``scipy.linalg.qr(pivoting=True)``)
pivots and ``|diag R|`` on tie-free inputs, and by the ID error bound.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

TIE_REL = 1e-12
NEAR_TIE_LOG = 1e-10


class NotSPD(Exception):
    """A Cholesky pivot was <= 0 (Remark 2.1: SPD lost)."""


def cholesky(a: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor; raises :class:`NotSPD` when a pivot is not positive."""
    if a.shape[0] == 0:
        return np.zeros((0, 0))
    if not np.all(np.isfinite(a)):
        raise NotSPD("non-finite block")
    try:
        return np.linalg.cholesky(a)
    except np.linalg.LinAlgError as e:
        raise NotSPD(str(e)) from None


def lsolve(Lf: np.ndarray, b: np.ndarray) -> np.ndarray:
    """L^{-1} b for lower-triangular L."""
    if Lf.shape[0] == 0:
        return np.zeros_like(b)
    return sla.solve_triangular(Lf, b, lower=True)


def ltsolve(Lf: np.ndarray, b: np.ndarray) -> np.ndarray:
    """L^{-T} b for lower-triangular L."""
    if Lf.shape[0] == 0:
        return np.zeros_like(b)
    return sla.solve_triangular(Lf, b, lower=True, trans="T")


def cpqr(M: np.ndarray, tol: float, log=None):
    """Column-pivoted Householder QR stopped at relative precision ``tol``.

    Returns ``(k, perm, R)``: ``perm`` lists original column indices in pivot
    order (the first ``k`` are the skeletons), ``R`` is the ``k x n`` leading
    block of the triangular factor in pivot order (``R[:, :k]`` upper
    triangular).
    """
    W = np.array(M, dtype=np.float64, copy=True)
    m, n = W.shape
    perm = np.arange(n)
    k = 0
    r11 = 0.0
    for j in range(min(m, n)):
        norms2 = np.einsum("ij,ij->j", W[j:, j:], W[j:, j:])
        mx = float(norms2.max())
        if j == 0:
            r11 = np.sqrt(mx)
            if r11 == 0.0:
                break
        if np.sqrt(mx) <= tol * r11:
            break
        cand = np.nonzero(norms2 >= (1.0 - TIE_REL) * mx)[0]
        p = j + cand[np.argmin(perm[j + cand])]
        if log is not None:
            near = np.nonzero(norms2 >= (1.0 - NEAR_TIE_LOG) * mx)[0]
            if near.size > 1:
                log.append((j, int(perm[p]), int(near.size)))
        if p != j:
            W[:, [j, p]] = W[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        x = W[j:, j].copy()
        nx = np.linalg.norm(x)
        alpha = -np.copysign(nx, x[0])
        v = x
        v[0] -= alpha
        beta = float(v @ v)
        if beta > 0.0 and j + 1 < n:
            W[j:, j + 1:] -= np.outer(v, (2.0 / beta) * (v @ W[j:, j + 1:]))
        W[j, j] = alpha
        W[j + 1:, j] = 0.0
        k = j + 1
    return k, perm, W[:k, :]


def interp_decomp(M: np.ndarray, tol: float, log=None):
    """ID of the columns of ``M`` (Sec. 2.2).

    Returns ``(k, perm, T)`` with ``M[:, perm[k:]] ~= M[:, perm[:k]] @ T``.
    """
    n = M.shape[1]
    k, perm, R = cpqr(M, tol, log)
    if k == 0:
        return 0, perm, np.zeros((0, n))
    T = sla.solve_triangular(R[:, :k], R[:, k:], lower=False)
    return k, perm, T
