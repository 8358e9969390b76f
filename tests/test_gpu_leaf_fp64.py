"""FP64 leaf fallback of the FP32 factor (precision pattern: leaf blocks whose
condition estimate exceeds a threshold are eliminated in FP64).

The GPU computes kappa_1(D A_II D), D = diag(A_II)^{-1/2}, of every 2D leaf
from its FP32 band factor: ||B||_1 from the stencil entries of L L^T and
||B^{-1}||_1 as the largest entry of B^{-1} 1 (B is an M-matrix, so B^{-1} is
entrywise nonnegative).  Checked against kappa_1 computed here with numpy on
the oracle's assembly: the flagged leaves are exactly those above the
threshold, up to the FP32 rounding of the band solves (kappa u_32 < 1e-2
here; a 10% band around the threshold is left open).  The re-eliminated
leaves bring the FP32 factor's F^{-1} closer to the FP64 factor's.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _exact_kappa1(A, n, m):
    """kappa_1(D A_II D) of every leaf (cell order: y major, x minor)."""
    A = A.tocsr()
    idx = np.arange(1, m)
    per = (n + 1) // m
    out = []
    for c in range(per * per):
        cy, cx = divmod(c, per)
        X, Y = np.meshgrid(cx * m + idx, cy * m + idx)
        g = ((X - 1) + n * (Y - 1)).ravel()
        B = A[g][:, g].toarray()
        s = 1.0 / np.sqrt(np.diag(B))
        B = B * s[:, None] * s[None, :]
        out.append(np.abs(B).sum(0).max() * np.abs(np.linalg.inv(B)).sum(0).max())
    return np.array(out)


@pytest.mark.parametrize("expo", [4, 5])
def test_flagged_leaves_bracket_the_exact_condition(gpu_lib, expo):
    ns, leaf = (255, 255), 16
    a = W.log_uniform_pixels(ns, 1e-4, 1e4, seed=W.SEED_BASE + 1)
    A = fd.assemble(ns, a, 0.0)
    k1 = _exact_kappa1(A, 255, leaf)
    thresh = 10.0 ** expo
    lo, hi = int(np.sum(k1 > 1.1 * thresh)), int(np.sum(k1 > thresh / 1.1))
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, leaf, 1e-3,
                             precision="fp32", leaf_fp64=expo)
    got = Fg.stats()["fp64_leaves"]
    print(f"\nleaf_fp64 1e{expo}: {got} leaves re-eliminated in FP64; exact kappa_1 above the "
          f"threshold / 1.1: {hi}, above 1.1 x threshold: {lo} (of {k1.size})")
    assert lo <= got <= hi
    f = _dev(W.normal_rhs(ns, 5))
    u, its, rr = Fg.pcg(f, rtol=1e-10)
    assert rr[0] <= 1.5e-10
    Fg.free()


def test_fp64_leaves_bring_the_fp32_factor_closer_to_fp64(gpu_lib):
    """All leaves re-eliminated (threshold 10): the FP32 factor's F^{-1} x
    moves towards the FP64 factor's, and the FP64 oracle's."""
    ns, leaf, tol = (127, 127), 16, 1e-6
    a = W.log_uniform_pixels(ns, 1e-4, 1e4, seed=W.SEED_BASE + 16 + 254)
    A = fd.assemble(ns, a, 0.0)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0)
    x = _dev(np.random.default_rng(8).standard_normal(A.shape[0]))
    y64 = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp64").apply(x).cpu().numpy()
    Fp = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp32", leaf_fp64=-1)
    Fa = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp32", leaf_fp64=1)
    assert Fp.stats()["fp64_leaves"] == 0
    assert Fa.stats()["fp64_leaves"] == 64
    dp = np.linalg.norm(Fp.apply(x).cpu().numpy() - y64) / np.linalg.norm(y64)
    da = np.linalg.norm(Fa.apply(x).cpu().numpy() - y64) / np.linalg.norm(y64)
    Ax = A @ x.cpu().numpy()
    Fo = phif.factor(A, ns, leaf, tol)
    eo = np.linalg.norm(phif.solve(Fo, Ax) - x.cpu().numpy()) / np.linalg.norm(x.cpu().numpy())
    ea = np.linalg.norm(Fa.apply(_dev(Ax)).cpu().numpy() - x.cpu().numpy()) / np.linalg.norm(x.cpu().numpy())
    print(f"\n127^2 tol 1e-6: |F32^-1x - F64^-1x|/|F64^-1x| plain {dp:.3e}, FP64 leaves {da:.3e}; "
          f"apply error with FP64 leaves {ea:.3e} (oracle {eo:.3e})")
    assert da < dp
    Fp.free()
    Fa.free()
