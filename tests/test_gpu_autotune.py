"""GPU tests of the scheduling autotuner (rhif_autotune).

The options it picks only split the work differently over CTAs, so the
factor they give must be the PHIF factor of the default schedule up to
rounding: the same skeletons (or, after an FP32 pivot flip, the same PCG
solution), and for FP64 the oracle's F^{-1} x.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _check_choice(kw):
    assert kw["big_front"] in (0, 1, -1)
    assert kw["big_frame"] in (0, 1, -1)
    assert kw["skel_cluster"] in (0, -1, 4)
    assert kw["tensor_cores"] in (0, -1)


def test_autotuned_fp64_factor_matches_oracle(gpu_lib):
    ns, leaf, tol = (31, 31, 31), 8, 1e-3
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=41)
    A = fd.assemble(ns, a, 1e-2)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 1e-2)
    kw, ms = gpu_lib.rhif_autotune(csr, ns, leaf, tol, precision="fp64", applies=10)
    assert ms > 0.0
    _check_choice(kw)
    Fg = gpu_lib.rhif_factor(csr, ns, leaf, tol, **kw)
    Fo = phif.factor(A, ns, leaf, tol)
    same = True
    for lvl in range(len(Fo.levels)):
        go = {frozenset(map(int, u.e)): frozenset(map(int, u.sk)) for u in Fo.levels[lvl].phases[0].units}
        gg = {frozenset(map(int, d)): frozenset(map(int, d[:k])) for d, k in Fg.skeletons(lvl, 0)}
        assert set(go) == set(gg)
        same &= go == gg
    assert same or Fo.ties
    if same:
        x = np.random.default_rng(43).standard_normal(A.shape[0])
        yg = Fg.apply(_dev(x)).cpu().numpy()
        yo = phif.solve(Fo, x)
        assert np.linalg.norm(yg - yo) <= 1e-9 * np.linalg.norm(yo)
    Fg.free()


def test_autotuned_fp32_factor_solves_like_the_default_schedule(gpu_lib):
    ns, leaf, tol = (255, 255), 8, 1e-3
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=44)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0)
    f = _dev(W.normal_rhs(ns, 45))
    kw, ms = gpu_lib.rhif_autotune(csr, ns, leaf, tol, precision="fp32", applies=10)
    assert ms > 0.0
    _check_choice(kw)
    tuned = gpu_lib.rhif_factor(csr, ns, leaf, tol, **kw)
    default = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp32")
    u1, _, r1 = tuned.pcg(f, rtol=1e-10)
    u0, _, r0 = default.pcg(f, rtol=1e-10)
    assert r1[0] <= 1.5e-10 and r0[0] <= 1.5e-10
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-7
    tuned.free()
    default.free()


def test_autotune_rejects_a_missing_output(gpu_lib):
    import ctypes
    ns = (15, 15)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(np.ones(W.pixel_shape(ns))), 0.0)
    rowptr, col, val = csr
    A = gpu_lib.CSR(rowptr.numel() - 1, val.numel(), rowptr.data_ptr(), col.data_ptr(),
                    val.data_ptr())
    rc = gpu_lib._lib.rhif_autotune(ctypes.byref(A), ctypes.byref(gpu_lib._grid(ns)), 4, 1e-3,
                                    None, 10, None, None, None)
    assert rc == -1   # RHIF_ERR_BAD_ARG
