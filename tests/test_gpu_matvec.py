"""The factor itself and its halves on the GPU (Eqs. 3.1 and 3.3): y = F x,
G^{-1} x and G^{-T} x with F = G G^T, and the Sec. 4 estimator
e_a = ||A - F|| / ||A||, against the FP64 oracle (phif.matvec, phif.apply_error).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [((63, 63), 8, 1e-3, (1e-3, 1e3), 0.0), ((63, 63), 8, 1e-6, (1e-4, 1e4), 0.0),
         ((15, 15, 15), 4, 1e-3, (1e-3, 1e3), 1e-2)]


@pytest.mark.parametrize("ns,leaf,tol,lohi,b", CASES)
def test_halves_compose_to_the_solve(gpu_lib, ns, leaf, tol, lohi, b):
    a = W.log_uniform_pixels(ns, *lohi, seed=sum(ns) + 7)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), b), ns, leaf, tol, precision="fp64")
    x = _dev(np.random.default_rng(3).standard_normal((2, Fg.N)))
    g = Fg.apply(x, op="half")
    y = Fg.apply(g, op="half_t")
    ref = Fg.apply(x)
    # the same launches in the same order: identical results
    np.testing.assert_array_equal(y.cpu().numpy(), ref.cpu().numpy())
    # ||G^{-1} x||^2 = x^T F^{-1} x
    for r in range(2):
        lhs = float(torch.dot(g[r], g[r]))
        rhs = float(torch.dot(x[r], ref[r]))
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    Fg.free()


@pytest.mark.parametrize("ns,leaf,tol,lohi,b", CASES)
def test_matvec_matches_oracle(gpu_lib, ns, leaf, tol, lohi, b):
    a = W.log_uniform_pixels(ns, *lohi, seed=sum(ns) + 7)
    A = fd.assemble(ns, a, b)
    Fo = phif.factor(A, ns, leaf, tol, edge_skel=len(ns) == 3)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), b), ns, leaf, tol, precision="fp64",
                             edge_skel_3d=len(ns) == 3)
    x = np.random.default_rng(4).standard_normal(A.shape[0])
    yg = Fg.matvec(_dev(x)).cpu().numpy()
    yo = phif.matvec(Fo, x)
    diff = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    back = np.linalg.norm(Fg.apply(_dev(yg)).cpu().numpy() - x) / np.linalg.norm(x)
    print(f"\nF x {ns} tol {tol:g}: |F x - F_oracle x| / |F_oracle x| = {diff:.2e}, "
          f"|F^-1 (F x) - x| / |x| = {back:.2e}")
    assert back <= 1e-12
    assert diff <= 1e-8
    Fg.free()


def test_matvec_is_A_at_tol_zero(gpu_lib):
    ns = (31, 31)
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=5)
    A = fd.assemble(ns, a, 0.0)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, 4, 0.0, precision="fp64")
    x = np.random.default_rng(6).standard_normal(A.shape[0])
    y = Fg.matvec(_dev(x)).cpu().numpy()
    assert np.linalg.norm(y - A @ x) <= 1e-10 * np.linalg.norm(A @ x)
    Fg.free()


@pytest.mark.parametrize("ns,leaf,tol", [((31, 31), 8, 1e-3), ((31, 31), 8, 1e-6), ((7, 7, 7), 4, 1e-2)])
def test_apply_error_estimate_matches_oracle(gpu_lib, ns, leaf, tol):
    """Same start vectors as the oracle's estimator (PCG64 seeds 0 and 1): the
    two power iterations agree to rounding."""
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=21)
    b = 1e-2 if len(ns) == 3 else 0.0
    A = fd.assemble(ns, a, b)
    Fo = phif.factor(A, ns, leaf, tol)
    n = A.shape[0]
    ea_o = phif.apply_error(A, Fo, seed=0)
    x0 = np.random.Generator(np.random.PCG64(0)).standard_normal(n)
    x1 = np.random.Generator(np.random.PCG64(1)).standard_normal(n)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), b), ns, leaf, tol, precision="fp64")
    ea_g, its = Fg.estimate_ea(_dev(x0), _dev(x1))
    print(f"\ne_a {ns} tol {tol:g}: gpu {ea_g:.6e} oracle {ea_o:.6e} ({its} products)")
    assert abs(ea_g - ea_o) <= 1e-6 * ea_o
    Fg.free()


def test_bad_operation_rejected(gpu_lib):
    import ctypes
    ns = (15, 15)
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=1)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, 4, 1e-3)
    x = _dev(np.ones(Fg.N))
    rc = gpu_lib._lib.rhif_apply(Fg._h, 4, 1, ctypes.c_void_p(x.data_ptr()), Fg.N,
                                 ctypes.c_void_p(x.data_ptr()), Fg.N, None)
    assert rc == -1
    rc = gpu_lib._lib.rhif_apply(Fg._h, 1, 1, ctypes.c_void_p(x.data_ptr()), Fg.N,
                                 ctypes.c_void_p(x.data_ptr()), Fg.N, None)
    assert rc == -1   # F x needs distinct x and y
    Fg.free()
