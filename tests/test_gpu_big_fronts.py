"""GPU tests of the many-CTA schedules for large fronts, frames and units.

A level whose fronts are large is eliminated by panel / trailing-tile / Schur-
tile launches spread over many CTAs, and its block Jacobi scaling (Eq. 2.3) by
row and column block solves; a skeletonization unit whose ID matrix is large
runs its CPQR on a thread-block cluster, one row slice per CTA.  Small objects
use one CTA each.  The thresholds and the cluster size are options, so these
tests force the many-CTA schedules on grids the oracle factors in seconds and
hold them to the same FP64 bar as the one-CTA schedule: identical skeletons
(except at logged near-ties) and F^{-1} x within 1e-9 relative of the oracle's.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [
    # ns, leaf, tol, b, edge
    ((63, 63), 8, 1e-6, 0.0, False),
    ((15, 15, 15), 4, 1e-3, 1e-2, False),
    ((11, 9, 13), 4, 1e-3, 1e-2, False),
    ((15, 15, 15), 4, 1e-3, 1e-2, True),
    ((31, 31, 31), 8, 1e-3, 1e-2, True),
]


_ORACLE = {}


def _oracle(ns, leaf, tol, b, edge):
    key = (ns, leaf, tol, b, edge)
    if key not in _ORACLE:
        a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=sum(ns) + leaf)
        A = fd.assemble(ns, a, b)
        _ORACLE[key] = (a, A, phif.factor(A, ns, leaf, tol, edge_skel=edge))
    return _ORACLE[key]


# skel_cluster: CTAs per skeletonization unit (thread-block cluster); 0 = default
# (one warp per small unit), -1 = one CTA per unit.
# The 31^3 grid runs with the default and one forced cluster size only.
PARAMS = [c + (k,) for c in CASES for k in ((0, 4) if c[0] == (31, 31, 31) else (0, -1, 1, 4, 16))]


@pytest.mark.parametrize("ns,leaf,tol,b,edge,skel_cluster", PARAMS)
def test_many_cta_schedules_match_oracle(gpu_lib, ns, leaf, tol, b, edge, skel_cluster):
    a, A, Fo = _oracle(ns, leaf, tol, b, edge)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), b)
    gpu_lib.rhif_reset_kernel_stats()
    Fg = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp64", edge_skel_3d=edge,
                             big_front=1, big_frame=1, skel_cluster=skel_cluster)
    ks = gpu_lib.rhif_kernel_stats()
    levels = Fg.stats()["levels"]
    # panel + trailing launches per 32 interior columns: more than one launch per level
    assert ks["partial_chol"]["launches"] > levels - 1
    # symmetrize + row products + column products on every preconditioned phase
    # (at least one per level below the root)
    assert ks["precond_scale"]["launches"] >= 3 * (levels - 1)
    same = True
    for lvl in range(len(Fo.levels)):
        for p in range(len(Fo.levels[lvl].phases)):
            go = {frozenset(map(int, u.e)): frozenset(map(int, u.sk))
                  for u in Fo.levels[lvl].phases[p].units}
            gg = {frozenset(map(int, d)): frozenset(map(int, d[:k])) for d, k in Fg.skeletons(lvl, p)}
            assert set(go) == set(gg)
            same &= go == gg
    assert same or Fo.ties
    x = np.random.default_rng(11).standard_normal(A.shape[0])
    yg = Fg.apply(_dev(x)).cpu().numpy()
    if same:
        yo = phif.solve(Fo, x)
        assert np.linalg.norm(yg - yo) <= 1e-9 * np.linalg.norm(yo)
    Fg.free()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_many_cta_schedules_agree_with_one_cta_schedule(gpu_lib, precision):
    """Same grid factored with the many-CTA schedules forced on and off: same
    skeletons, F^{-1} x equal to rounding, PCG converges to the same solution."""
    ns, leaf = (31, 31, 31), 8
    a = W.log_uniform_pixels(ns, 1e-4, 1e4, seed=21)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0)
    f = _dev(W.normal_rhs(ns, 22))
    on = gpu_lib.rhif_factor(csr, ns, leaf, 1e-3, precision=precision, big_front=1, big_frame=1)
    off = gpu_lib.rhif_factor(csr, ns, leaf, 1e-3, precision=precision, big_front=-1, big_frame=-1)
    lv = on.stats()["levels"]
    sk_on = [on.skeletons(l, p) for l in range(lv) for p in range(1)]
    sk_off = [off.skeletons(l, p) for l in range(lv) for p in range(1)]
    eps = 1e-12 if precision == "fp64" else 1e-4
    if sk_on == sk_off:
        y1 = on.apply(f)
        y0 = off.apply(f)
        assert float(torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)) <= eps
    u1, _, r1 = on.pcg(f, rtol=1e-10)
    u0, _, r0 = off.pcg(f, rtol=1e-10)
    assert r1[0] <= 1.5e-10 and r0[0] <= 1.5e-10
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-8
    on.free()
    off.free()


def test_tensor_core_schur_agrees_with_cuda_cores(gpu_lib):
    """FP32 factor with the Schur complements of the large fronts on the
    tensor cores (3xTF32) vs on the CUDA cores: F^{-1} x agrees to FP32-level
    rounding when the skeletons coincide, and PCG reaches the same solution."""
    ns, leaf = (31, 31, 31), 8
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=33)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 1e-2)
    f = _dev(W.normal_rhs(ns, 34))
    kw = dict(precision="fp32", edge_skel_3d=True, big_front=1, big_frame=1)
    on = gpu_lib.rhif_factor(csr, ns, leaf, 1e-3, tensor_cores=0, **kw)
    off = gpu_lib.rhif_factor(csr, ns, leaf, 1e-3, tensor_cores=-1, **kw)
    lv = on.stats()["levels"]
    if [on.skeletons(l) for l in range(lv)] == [off.skeletons(l) for l in range(lv)]:
        y1, y0 = on.apply(f), off.apply(f)
        assert float(torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)) <= 1e-4
    u1, _, r1 = on.pcg(f, rtol=1e-10)
    u0, _, r0 = off.pcg(f, rtol=1e-10)
    assert r1[0] <= 1.5e-10 and r0[0] <= 1.5e-10
    assert float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)) <= 1e-8
    on.free()
    off.free()
