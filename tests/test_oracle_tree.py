"""Pins of the oracle's grouping (Sec. 3.1 Fig. 3, Sec. 3.2) against closed forms.

The oracle classifies each DOF through a per-axis key; these tests rebuild the
expected groups from a different description — products of per-axis runs of
grid points (cell interiors along an axis, and separator planes) — and from the
per-level counts and sizes the paper states (2D: cells, edges, corners; 3D:
cells, faces, edges, corners, with the face size read as (2^l m - 1)^2), so
that a misclassified group (a wrong type, a node in the wrong cell, a group
split or merged) changes a count or a size.
"""
import itertools

import numpy as np
import pytest

from oracle import tree


def _axis_runs(n, w):
    """Per axis: cell interiors as (kind 'i', cell index, length) and separator
    planes as (kind 'p', plane index, 1), for interior nodes 1..n and cell width w."""
    runs = []
    ncell = -(-(n + 1) // w)
    for c in range(ncell):
        lo, hi = c * w + 1, min(c * w + w - 1, n)
        if hi >= lo:
            runs.append(("i", c, hi - lo + 1))
        q = (c + 1) * w
        if q <= n:
            runs.append(("p", c + 1, 1))
    return runs


def _closed_form_groups(ns, w):
    """{type t: sorted list of group sizes} for ALL interior nodes of the grid,
    t = number of axes on which the group lies on a separator plane."""
    out = {}
    for combo in itertools.product(*[_axis_runs(n, w) for n in ns]):
        t = sum(1 for r in combo if r[0] == "p")
        size = int(np.prod([r[2] for r in combo]))
        out.setdefault(t, []).append(size)
    return {t: sorted(v) for t, v in out.items()}


def _oracle_groups(ns, gids, w):
    out = {}
    for key, t, mem in tree.groups(ns, gids, w):
        out.setdefault(t, []).append(int(mem.size))
    return {t: sorted(v) for t, v in out.items()}


@pytest.mark.parametrize("ns,leaf", [((127, 127), 8), ((1023, 1023), 16), ((20, 23), 4),
                                     ((63, 63, 63), 8), ((11, 9, 13), 4), ((1, 5), 2)])
def test_level0_groups_match_per_axis_product_form(ns, leaf):
    N = int(np.prod(ns))
    got = _oracle_groups(ns, np.arange(N), leaf)
    want = _closed_form_groups(ns, leaf)
    assert got == want
    assert sum(sum(v) for v in got.values()) == N


def test_level0_counts_stated_for_the_benchmark_grids():
    # 127^2, leaf 8: 256 cells of 49, 480 edges of 7, 225 corners
    g = _oracle_groups((127, 127), np.arange(127 * 127), 8)
    assert g[0] == [49] * 256 and g[1] == [7] * 480 and g[2] == [1] * 225
    assert 256 * 49 + 480 * 7 + 225 == 16129
    # 1023^2, leaf 16: 4096 cells of 225, 8064 edges of 15, 3969 corners
    g = _oracle_groups((1023, 1023), np.arange(1023 * 1023), 16)
    assert g[0] == [225] * 4096 and g[1] == [15] * 8064 and g[2] == [1] * 3969
    # 63^3, leaf 8: 512 cells of 343, 1344 faces of 49, 1176 edges of 7, 343 corners
    g = _oracle_groups((63, 63, 63), np.arange(63 ** 3), 8)
    assert g[0] == [343] * 512 and g[1] == [49] * 1344 and g[2] == [7] * 1176 and g[3] == [1] * 343
    assert 512 * 343 + 1344 * 49 + 1176 * 7 + 343 == 250047


def _separator_survivors(ns, w_prev):
    """DOFs on a separator of the previous level (cell width w_prev): the
    active set after level l-1 when every separator DOF is kept (tol = 0)."""
    N = int(np.prod(ns))
    x = tree.coords(ns, np.arange(N))
    return np.nonzero(np.any(x % w_prev == 0, axis=1))[0]


@pytest.mark.parametrize("ns,leaf", [((127, 127), 8), ((63, 63), 4)])
def test_upper_levels_2d_match_stated_sizes(ns, leaf):
    """Level l >= 1, 2D, every separator DOF kept (edge rank k = 2^(l-1) m - 1):
    4^(L-l) cells with |I| = 4k + 1, 2(2^(L-l) - 1) 2^(L-l) edges of 2k + 1,
    (2^(L-l) - 1)^2 corners."""
    L = tree.num_levels(ns, leaf)
    for l in range(1, L + 1):
        k = (1 << (l - 1)) * leaf - 1
        q = 1 << (L - l)
        g = _oracle_groups(ns, _separator_survivors(ns, (1 << (l - 1)) * leaf), (1 << l) * leaf)
        assert g[0] == [4 * k + 1] * (q * q)
        assert g.get(1, []) == [2 * k + 1] * (2 * (q - 1) * q)
        assert g.get(2, []) == [1] * ((q - 1) ** 2)


@pytest.mark.parametrize("ns,leaf", [((63, 63, 63), 8), ((31, 31, 31), 4)])
def test_upper_levels_3d_match_stated_sizes(ns, leaf):
    """Level l >= 1, 3D, every separator DOF kept (half-face k_f = (2^(l-1) m - 1)^2):
    8^(L-l) cells with |I| = 12 k_f + 6 (2^(l-1) m - 1) + 1, faces of
    4 k_f + 4 (2^(l-1) m - 1) + 1 = (2^l m - 1)^2, edges of 2^l m - 1."""
    L = tree.num_levels(ns, leaf)
    for l in range(1, L + 1):
        e = (1 << (l - 1)) * leaf - 1
        kf = e * e
        q = 1 << (L - l)
        g = _oracle_groups(ns, _separator_survivors(ns, (1 << (l - 1)) * leaf), (1 << l) * leaf)
        assert g[0] == [12 * kf + 6 * e + 1] * q ** 3
        assert g.get(1, []) == [4 * kf + 4 * e + 1] * (3 * (q - 1) * q * q)
        assert (4 * kf + 4 * e + 1) == ((1 << l) * leaf - 1) ** 2
        assert g.get(2, []) == [(1 << l) * leaf - 1] * (3 * (q - 1) ** 2 * q)
        assert g.get(3, []) == [1] * ((q - 1) ** 3)


@pytest.mark.parametrize("ns,leaf", [((20, 23), 4), ((11, 9, 13), 4), ((15, 15), 4)])
def test_cells_of_key_is_every_cell_whose_closure_holds_the_group(ns, leaf):
    """cells_of_key against brute force: a cell (c_1..c_d) holds a node x when
    c_i w <= x_i <= (c_i + 1) w on every axis; the cells of a group are those
    holding all of its nodes, within the padded tree."""
    L = tree.num_levels(ns, leaf)
    for l in range(L):
        w = (1 << l) * leaf
        ncell = 1 << (L - l)
        for key, t, mem in tree.groups(ns, np.arange(int(np.prod(ns))), w):
            x = tree.coords(ns, mem)
            brute = []
            for c in itertools.product(range(ncell), repeat=len(ns)):
                c = tuple(c)
                if all(np.all((c[i] * w <= x[:, i]) & (x[:, i] <= (c[i] + 1) * w)) for i in range(len(ns))):
                    brute.append(c)
            assert sorted(tree.cells_of_key(key)) == sorted(brute)
            assert len(brute) == 2 ** t


def test_groups_ignore_inactive_dofs_and_sort_members():
    ns, leaf = (15, 15), 4
    rng = np.random.default_rng(3)
    act = np.sort(rng.choice(225, 120, replace=False))
    for key, t, mem in tree.groups(ns, rng.permutation(act), leaf):
        assert np.all(np.diff(mem) > 0)
        assert np.isin(mem, act).all()
    got = np.sort(np.concatenate([m for _, _, m in tree.groups(ns, act, leaf)]))
    np.testing.assert_array_equal(got, act)
