"""Quadtree/octree grouping of the DOFs (Sec. 3.1, Fig. 3; Sec. 3.2).

Grid: ``n = 2^L m`` intervals per axis (``m`` = leaf width); interior nodes
have 1-based coordinates ``1..n-1``.  At level ``l`` the cells are
``2^l m`` intervals wide.  A node whose coordinates contain ``t`` multiples of
the cell width lies on a separator of type ``t``: ``t = 0`` is a cell interior,
``t = 1`` an edge (2D) or face (3D), ``t = 2`` a corner (2D) or edge (3D),
``t = 3`` a corner (3D).  Only still-active DOFs are grouped; the members of a
group are listed in ascending global index.

Grids whose side is not of the form ``2^L m - 1`` are handled by padding the
tree: ``L`` is the smallest level count with ``2^L m >= n_i + 1`` on every
axis, and the nodes beyond the grid simply do not exist (reading of Sec. 3.1
for general sizes).
"""
from __future__ import annotations

import numpy as np


def num_levels(ns, leaf: int) -> int:
    """Smallest L with 2^L * leaf >= n_i + 1 for every axis."""
    need = max(int(n) + 1 for n in ns)
    L = 0
    while leaf * (1 << L) < need:
        L += 1
    return L


def coords(ns, gids: np.ndarray) -> np.ndarray:
    """1-based node coordinates, shape (len(gids), d), x first."""
    gids = np.asarray(gids, dtype=np.int64)
    out = np.empty((gids.size, len(ns)), dtype=np.int64)
    rem = gids.copy()
    for ax, n in enumerate(ns):
        out[:, ax] = rem % n + 1
        rem //= n
    return out


def group_keys(ns, gids: np.ndarray, width: int):
    """Per-DOF group key at cell width ``width``.

    Along each axis ``v = 2*(x // width) + (x % width != 0)``: odd ``v`` means
    inside cell ``(v-1)/2``; even ``v`` means on the plane between cells
    ``v/2 - 1`` and ``v/2``.  Returns (keys (len, d), type t = number of even v).
    """
    x = coords(ns, gids)
    v = 2 * (x // width) + (x % width != 0)
    t = np.sum(v % 2 == 0, axis=1)
    return v, t


def groups(ns, gids: np.ndarray, width: int):
    """Group the active DOFs ``gids`` at cell width ``width``.

    Returns a list of ``(key tuple, type t, member gids ascending)`` sorted by
    key (x-major lexicographic on the key tuple read from the last axis).
    """
    gids = np.sort(np.asarray(gids, dtype=np.int64))
    if gids.size == 0:
        return []
    v, t = group_keys(ns, gids, width)
    d = len(ns)
    base = int(v.max()) + 1
    code = np.zeros(gids.size, dtype=np.int64)
    for ax in reversed(range(d)):
        code = code * base + v[:, ax]
    order = np.lexsort((gids, code))
    code_s = code[order]
    cut = np.nonzero(np.diff(code_s))[0] + 1
    out = []
    for chunk in np.split(order, cut):
        key = tuple(int(q) for q in v[chunk[0]])
        out.append((key, int(t[chunk[0]]), gids[chunk]))
    return out


def cells_of_key(key) -> list:
    """Cells (index tuples, x first) whose closure contains the group ``key``."""
    choices = []
    for v in key:
        if v % 2:
            choices.append([(v - 1) // 2])
        else:
            choices.append([v // 2 - 1, v // 2])
    out = [()]
    for ch in choices:
        out = [o + (c,) for o in out for c in ch]
    return out
