"""Finite-difference matrix of -div(a grad u) + b u on the unit square/cube.

Eq. (1.1) discretised as in Sec. 3.1 (five-point stencil, 2D) and Sec. 3.2
(seven-point stencil, 3D) on a uniform grid with zero Dirichlet data; the DOFs
are the interior node values, giving the sparse SPD system of Eq. (1.2).

The paper does not print the stencil weights for a variable coefficient.
Reading used here: the coefficient is constant on each grid pixel (voxel); the
weight of the grid edge between two neighbouring nodes is the arithmetic mean
of ``a`` over the 2 (2D) or 4 (3D) pixels that touch that edge; an edge to a
boundary node only adds to the diagonal; ``h_i = 1/(n_i + 1)`` per axis and the
``1/h^2`` factor is kept; ``b`` is added to the diagonal unscaled.

Parity: pinned by the closed-form sine spectrum of the constant-coefficient
Laplacian, by the pixel-wise energy identity and by a hand-worked 2x2 fixture.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _edge_weights(a: np.ndarray, d: int, ax: int) -> np.ndarray:
    """Mean of ``a`` over the pixels touching each grid edge parallel to axis ``ax``.

    ``a`` has C-order shape (..., ny+1, nx+1); axis ``ax`` (0 = x) is array
    axis ``d-1-ax``.  The result has ``n_ax + 1`` entries along ``ax`` (edge
    from node coordinate x to x+1, x = 0..n_ax) and ``n_o`` along every other
    axis (node coordinates 1..n_o).
    """
    w = a
    for o in range(d):
        if o == ax:
            continue
        arr_axis = d - 1 - o
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[arr_axis] = slice(0, -1)
        hi[arr_axis] = slice(1, None)
        w = 0.5 * (w[tuple(lo)] + w[tuple(hi)])
    return w


def assemble(ns, a_pix: np.ndarray, b=0.0) -> sp.csr_matrix:
    """Sparse FP64 matrix A of Eq. (1.2); rows/cols in DOF order (x fastest)."""
    ns = tuple(int(n) for n in ns)
    d = len(ns)
    a_pix = np.asarray(a_pix, dtype=np.float64)
    assert a_pix.shape == tuple(n + 1 for n in reversed(ns))
    node_shape = tuple(reversed(ns))
    N = int(np.prod(ns))
    ids = np.arange(N).reshape(node_shape)
    diag = np.zeros(node_shape)
    rows, cols, vals = [], [], []
    for ax in range(d):
        h = 1.0 / (ns[ax] + 1)
        arr_axis = d - 1 - ax
        w = _edge_weights(a_pix, d, ax) / (h * h)
        n = ns[ax]
        left = [slice(None)] * d
        right = [slice(None)] * d
        left[arr_axis] = slice(0, n)        # edge from node coordinate x-1 to x
        right[arr_axis] = slice(1, n + 1)   # edge from x to x+1
        diag += w[tuple(left)] + w[tuple(right)]
        inner = [slice(None)] * d
        inner[arr_axis] = slice(1, n)       # edges between two interior nodes
        wi = w[tuple(inner)]
        lo_ids = [slice(None)] * d
        hi_ids = [slice(None)] * d
        lo_ids[arr_axis] = slice(0, n - 1)
        hi_ids[arr_axis] = slice(1, n)
        r = ids[tuple(lo_ids)].ravel()
        c = ids[tuple(hi_ids)].ravel()
        v = -wi.ravel()
        rows += [r, c]
        cols += [c, r]
        vals += [v, v]
    if np.isscalar(b):
        diag = diag + float(b)
    else:
        diag = diag + np.asarray(b, dtype=np.float64).reshape(node_shape)
    rows.append(ids.ravel())
    cols.append(ids.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def dA_dlog_a(ns, a_pix: np.ndarray, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Per-pixel ``-lam^T (dA/d log a_p) u`` for the assembly above.

    A is linear in ``a``: pixel p contributes ``a_p / 2^(d-1)`` to the weight
    of each of its grid edges, so
    ``d(lam^T A u)/d log a_p = a_p/2^(d-1) * sum_{edges e of p} (lam_i-lam_j)(u_i-u_j)/h_e^2``
    with ``lam = u = 0`` on boundary nodes.  Returns the negated sum, i.e. the
    gradient of ``0.5||u - u_obs||^2`` when ``lam = A^{-1}(u - u_obs)``.
    """
    ns = tuple(int(n) for n in ns)
    d = len(ns)
    node_shape = tuple(reversed(ns))
    U = np.zeros(tuple(n + 2 for n in node_shape))
    Lm = np.zeros_like(U)
    U[tuple(slice(1, -1) for _ in range(d))] = np.asarray(u).reshape(node_shape)
    Lm[tuple(slice(1, -1) for _ in range(d))] = np.asarray(lam).reshape(node_shape)
    grad = np.zeros_like(a_pix, dtype=np.float64)
    for ax in range(d):
        h = 1.0 / (ns[ax] + 1)
        arr_axis = d - 1 - ax
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[arr_axis] = slice(0, -1)
        hi[arr_axis] = slice(1, None)
        du = U[tuple(hi)] - U[tuple(lo)]
        dl = Lm[tuple(hi)] - Lm[tuple(lo)]
        prod = du * dl / (h * h)   # per grid edge parallel to ax, padded node grid
        # every pixel p touches the edges parallel to ax at its 2^(d-1) "corners"
        # in the other axes; sum those edge products into the pixel.
        for mask in range(1 << (d - 1)):
            sl = [slice(None)] * d
            bit = 0
            for o in range(d):
                if o == ax:
                    continue
                oa = d - 1 - o
                sl[oa] = slice(1, None) if (mask >> bit) & 1 else slice(0, -1)
                bit += 1
            grad += prod[tuple(sl)]
    return -a_pix * grad / (1 << (d - 1))
