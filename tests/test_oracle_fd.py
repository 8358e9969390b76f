"""Pins for the oracle's finite-difference matrix (Eqs. 1.1-1.2, Sec. 3.1, Sec. 3.2)."""
import itertools
import os

import numpy as np
import pytest

import workloads as W
from oracle import fd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_worked_2x2_fixture():
    lines = [ln.split() for ln in open(os.path.join(GOLDEN, "fd_2x2.txt")) if ln.strip() and ln[0] != "#"]
    pix = np.array([float(v) for v in lines[0][1:]]).reshape(3, 3)
    rows = np.array([[float(v) for v in ln[1:]] for ln in lines[1:]])
    A = fd.assemble((2, 2), pix, 0.0).toarray()
    np.testing.assert_allclose(A, rows, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ns", [(9, 9), (15, 7), (5, 6, 7)])
def test_constant_coefficient_sine_spectrum(ns):
    """a = 1, b = 0: sin modes are eigenvectors with the closed-form eigenvalues
    sum_i (4/h_i^2) sin^2(j_i pi h_i / 2)."""
    d = len(ns)
    a = np.ones(W.pixel_shape(ns))
    A = fd.assemble(ns, a, 0.0)
    hs = [1.0 / (n + 1) for n in ns]
    xs = [np.arange(1, n + 1) * h for n, h in zip(ns, hs)]
    rng = np.random.default_rng(3)
    for _ in range(6):
        js = [int(rng.integers(1, n + 1)) for n in ns]
        grids = np.meshgrid(*reversed(xs), indexing="ij")[::-1]
        v = np.ones(grids[0].shape)
        for ax in range(d):
            v = v * np.sin(js[ax] * np.pi * grids[ax])
        v = v.ravel()
        lam = sum(4.0 / hs[ax] ** 2 * np.sin(js[ax] * np.pi * hs[ax] / 2) ** 2 for ax in range(d))
        np.testing.assert_allclose(A @ v, lam * v, rtol=0, atol=1e-11 * lam * np.abs(v).max())


def _energy_by_pixels(ns, a, b, u):
    """sum_p a_p / 2^(d-1) * sum_{grid edges of pixel p} (du)^2 / h^2 + sum b u^2,
    written as plain loops over pixels with u = 0 on the boundary."""
    d = len(ns)
    node = np.zeros(tuple(n + 2 for n in reversed(ns)))
    node[tuple(slice(1, -1) for _ in range(d))] = u.reshape(tuple(reversed(ns)))
    total = 0.0
    for p in itertools.product(*[range(n + 1) for n in reversed(ns)]):  # (z,) y, x
        corners = list(itertools.product(*[(c, c + 1) for c in p]))
        for c0 in corners:
            for ax in range(d):
                arr_ax = d - 1 - ax
                if c0[arr_ax] != p[arr_ax]:
                    continue
                c1 = list(c0)
                c1[arr_ax] += 1
                h = 1.0 / (ns[ax] + 1)
                du = node[tuple(c1)] - node[c0]
                total += a[p] / 2 ** (d - 1) * du * du / (h * h)
    return total + float(np.sum(b * u * u))


@pytest.mark.parametrize("ns,b", [((4, 5), 0.0), ((3, 4, 3), 0.37)])
def test_energy_identity(ns, b):
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=7)
    A = fd.assemble(ns, a, b)
    u = np.random.default_rng(1).standard_normal(A.shape[0])
    e1 = float(u @ (A @ u))
    e2 = _energy_by_pixels(ns, a, b, u)
    assert abs(e1 - e2) <= 1e-12 * abs(e2)
    assert (A - A.T).nnz == 0 or abs(A - A.T).max() == 0.0


def test_gradient_formula_matches_finite_differences():
    """d/dlog a_p of 0.5||A^{-1}f - u_obs||^2 via the adjoint formula vs central FD."""
    import scipy.sparse.linalg as spla
    ns = (5, 4)
    la = np.log(W.log_uniform_pixels(ns, 1e-1, 1e1, seed=2))
    f = W.normal_rhs(ns, 3)
    u_obs = W.normal_rhs(ns, 4)

    def loss(la_):
        A = fd.assemble(ns, np.exp(la_), 0.0).tocsc()
        u = spla.spsolve(A, f)
        return 0.5 * float(np.sum((u - u_obs) ** 2))

    A = fd.assemble(ns, np.exp(la), 0.0).tocsc()
    u = spla.spsolve(A, f)
    lam = spla.spsolve(A, u - u_obs)
    g = fd.dA_dlog_a(ns, np.exp(la), u, lam)
    delta = 1e-5
    for idx in [(0, 0), (2, 3), (4, 5), (1, 2)]:
        e = np.zeros_like(la)
        e[idx] = delta
        fdg = (loss(la + e) - loss(la - e)) / (2 * delta)
        assert abs(fdg - g[idx]) <= 1e-6 * max(1.0, abs(fdg))
