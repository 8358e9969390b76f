"""The diagonal local preconditioner (concluding section: any local
preconditioner, e.g. diagonal, may replace block Cholesky) on the GPU against
the FP64 oracle with the same option.

C_g = diag(A_gg)^{-1/2} for every separator group; everything else is the PHIF
factorization of Sec. 3.  FP64 bar as for block Jacobi: identical skeleton
sets except at logged ties, F^{-1} x within 1e-9 of the oracle's, apply error
within 2x of the oracle's; the FP32 factor with this option still drives PCG
to relres 1e-10.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _skeleton_map(units):
    return {frozenset(int(g) for g in dofs): frozenset(int(g) for g in dofs[:k]) for dofs, k in units}


CASES = [
    ((31, 31), 8, 1e-3, (1e-3, 1e3), 0.0, False),
    ((63, 63), 8, 1e-6, (1e-4, 1e4), 0.0, False),
    ((127, 127), 16, 1e-3, (1e-4, 1e4), 0.0, False),
    ((20, 23), 4, 1e-3, (1e-2, 1e2), 0.0, False),
    ((15, 15, 15), 4, 1e-3, (1e-3, 1e3), 1e-2, True),
]


@pytest.mark.parametrize("ns,leaf,tol,lohi,b,edge", CASES)
def test_diag_precond_fp64_matches_oracle(gpu_lib, ns, leaf, tol, lohi, b, edge):
    a = W.log_uniform_pixels(ns, *lohi, seed=sum(ns) + 3 * leaf)
    A = fd.assemble(ns, a, b)
    Fo = phif.factor(A, ns, leaf, tol, precondition="diag", edge_skel=edge)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), b), ns, leaf, tol,
                             precision="fp64", precondition="diag", edge_skel_3d=edge)
    diverged = False
    for lvl in range(len(Fo.levels)):
        for ph in range(len(Fo.levels[lvl].phases)):
            go = {frozenset(int(g) for g in u.e): frozenset(int(g) for g in u.sk)
                  for u in Fo.levels[lvl].phases[ph].units}
            gg = _skeleton_map(Fg.skeletons(lvl, ph))
            assert set(go) == set(gg)
            if any(go[u] != gg[u] for u in go):
                assert Fo.ties, f"skeleton sets differ at level {lvl} phase {ph} without a logged tie"
                diverged = True
        if diverged:
            break
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    yg = Fg.apply(_dev(x)).cpu().numpy()
    yo = phif.solve(Fo, x)
    diff = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    Ax = A @ x
    eg = np.linalg.norm(Fg.apply(_dev(Ax)).cpu().numpy() - x) / np.linalg.norm(x)
    eo = np.linalg.norm(phif.solve(Fo, Ax) - x) / np.linalg.norm(x)
    print(f"\ndiag precond {ns} leaf {leaf} tol {tol:g}: diff {diff:.2e}, apply err gpu {eg:.3e} "
          f"oracle {eo:.3e}")
    if not diverged:
        assert Fg.stats()["root_size"] == Fo.S.size
        assert diff <= 1e-9
    assert eg <= 2 * eo + 1e-12
    Fg.free()


def test_diag_precond_fp32_pcg(gpu_lib):
    ns = (255, 255)
    a = W.log_uniform_pixels(ns, 1e-4, 1e4, seed=77)
    A = fd.assemble(ns, a, 0.0)
    f = W.normal_rhs(ns, 78)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0)
    its = {}
    for mode in ("none", "diag", "block"):
        Fg = gpu_lib.rhif_factor(csr, ns, 16, 1e-3, precision="fp32", precondition=mode)
        u, it, rr = Fg.pcg(_dev(f), rtol=1e-10, maxit=500)
        assert rr[0] <= 1.5e-10
        ud = spla.spsolve(A.tocsc(), f)
        assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-6 * np.linalg.norm(ud)
        its[mode] = it[0]
        Fg.free()
    print(f"\n255^2 fp32 PCG iterations by local preconditioner: {its}")
    assert its["block"] <= its["diag"] <= its["none"]

