"""Pins for the oracle's PCG (Sec. 4: PCG with F^{-1} as the preconditioner).

What the mathematics fixes, independently of the factorization:
  * with an exact preconditioner (the factor at tol = 0 is A itself, Sec. 3)
    the first PCG step already solves the system;
  * CG on a right-hand side with components along m eigenvectors of distinct
    eigenvalues terminates after m steps (Krylov space of dimension m); the
    sine modes are the eigenvectors of the constant-coefficient Laplacian;
  * on a generic right-hand side, plain CG stays within the classical bound
    k <= ceil(sqrt(kappa)/2 * ln(2/eps)) with kappa = cot^2(pi h / 2) for the
    5-point Laplacian with Dirichlet boundary.
A wrong step length, a wrong beta or a stale residual breaks one of them.
"""
import math

import numpy as np

import workloads as W
from oracle import fd, phif


def _laplacian(n):
    ns = (n, n)
    return ns, fd.assemble(ns, np.ones(W.pixel_shape(ns)), 0.0)


def _mode(n, j, k):
    h = 1.0 / (n + 1)
    xs = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(xs, xs)
    return (np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)).ravel()


def test_exact_factor_makes_pcg_converge_in_one_step():
    ns = (31, 31)
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=51)
    A = fd.assemble(ns, a, 0.0)
    F = phif.factor(A, ns, 4, 0.0)
    f = W.normal_rhs(ns, 52)
    u, it, rr = phif.pcg(A, f, M=lambda r: phif.solve(F, r), rtol=1e-10)
    assert it == 1
    assert rr <= 1e-12


def test_cg_terminates_after_as_many_steps_as_distinct_eigenvalues():
    n = 31
    ns, A = _laplacian(n)
    f1 = _mode(n, 3, 4)                       # one eigenvector: one step
    _, it1, rr1 = phif.pcg(A, f1, rtol=1e-10)
    assert it1 == 1 and rr1 <= 1e-12
    # three eigenvalues (modes (3,4) and (4,3) share one, so four modes give three)
    f3 = _mode(n, 3, 4) + 0.5 * _mode(n, 4, 3) - 2.0 * _mode(n, 1, 1) + _mode(n, 20, 7)
    _, it3, rr3 = phif.pcg(A, f3, rtol=1e-10)
    assert it3 == 3 and rr3 <= 1e-11


def test_plain_cg_within_the_classical_bound_on_the_laplacian():
    for n in (31, 63):
        ns, A = _laplacian(n)
        h = 1.0 / (n + 1)
        kappa = 1.0 / math.tan(math.pi * h / 2) ** 2
        eps = 1e-8
        # the bound is on the A-norm of the error; the residual 2-norm picks up
        # at most a factor sqrt(kappa), so bound it at eps / sqrt(kappa)
        bound = math.ceil(0.5 * math.sqrt(kappa) * math.log(2 * math.sqrt(kappa) / eps))
        f = W.normal_rhs(ns, 53 + n)
        _, it, rr = phif.pcg(A, f, rtol=eps)
        assert rr <= 2 * eps
        assert it <= bound
        assert it >= 0.25 * math.sqrt(kappa)   # a random f excites the whole spectrum
