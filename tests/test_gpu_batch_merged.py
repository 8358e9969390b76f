"""Merged batches (rhif_factor_batch): the cells, groups and units of every
problem at a level form one work list, one launch per level step for the
whole batch (cells, block-Jacobi steps and the IDs of a level commute,
Secs. 2.1-2.3, and the problems share nothing).

The bar: every problem of the batch gets the factor it gets alone — the same
unit sets and skeleton sets at every level, F^{-1} x equal to the single
problem's up to rounding order (the merged level may pick another kernel
variant from the batch's largest block sizes), the same PCG iteration counts
and solutions; and the FP64 batch against the FP64 oracle on one problem.
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


def _problems(sides, d=2, lohi=(1e-3, 1e3), seed=300):
    out = []
    for i, s in enumerate(sides):
        ns = (s,) * d if np.isscalar(s) else tuple(s)
        a = W.log_uniform_pixels(ns, *lohi, seed=seed + i)
        out.append((ns, a))
    return out


def _skel_sets(units, lo, hi):
    """{unit dofs: skeleton dofs} of the units lying in DOF range [lo, hi), local numbering."""
    out = {}
    for dofs, k in units:
        if lo <= dofs[0] < hi:
            out[frozenset(int(g) - lo for g in dofs)] = frozenset(int(g) - lo for g in dofs[:k])
    return out


def _check_against_singles(lib, probs, leaf, tol, precision, b=0.0, edge=False, rel=1e-12):
    csrs = [lib.rhif_assemble_fd(ns, _dev(a), b) for ns, a in probs]
    grids = [ns for ns, _ in probs]
    FB = lib.rhif_factor_batch(csrs, grids, leaf, tol, precision=precision, edge_skel_3d=edge)
    rng = np.random.default_rng(17)
    xs = [rng.standard_normal(int(np.prod(ns))) for ns in grids]
    yb = FB.apply(_dev(np.concatenate(xs))).cpu().numpy()
    stb = FB.stats()
    for i, ((ns, a), csr) in enumerate(zip(probs, csrs)):
        F = lib.rhif_factor(csr, ns, leaf, tol, precision=precision, edge_skel_3d=edge)
        st = F.stats()
        lo, hi = FB.dof_base[i], FB.dof_base[i + 1]
        # FP32 pivots may flip where two column norms agree to FP32 rounding
        # and the merged level runs another kernel variant; FP64 ones may not
        for lvl in range(st["levels"] if precision == "fp64" else 0):
            for ph in range(2 if edge else 1):
                single = _skel_sets(F.skeletons(lvl, ph), 0, hi - lo)
                merged = _skel_sets(FB.skeletons(lvl, ph), lo, hi)
                assert single == merged, f"problem {i} level {lvl} phase {ph}"
        y = F.apply(_dev(xs[i])).cpu().numpy()
        diff = np.linalg.norm(yb[lo:hi] - y) / np.linalg.norm(y)
        assert diff <= rel, f"problem {i}: F^-1 x differs by {diff:.2e}"
        F.free()
    assert stb["levels"] == max(lib.rhif_factor(c, ns, leaf, tol).stats()["levels"]
                                for c, ns in zip(csrs, grids))
    return FB, csrs, grids


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_merged_batch_2d_matches_single_problems(gpu_lib, precision):
    # sides give 2 to 5 levels at leaf 8: roots on four different merged levels
    probs = _problems([31, 47, 64, 70, 39, 20, 130, 255])
    FB, csrs, grids = _check_against_singles(gpu_lib, probs, 8, 1e-3, precision,
                                             rel=1e-12 if precision == "fp64" else 1e-3)
    # PCG: per-problem right-hand-side blocks, 3 right-hand sides each
    fs = [_dev(W.normal_rhs(ns, 400 + i, nrhs=3)) for i, ns in enumerate(grids)]
    us, its, rr = FB.pcg_batch(fs, rtol=1e-10)
    for i, (ns, a) in enumerate(probs):
        A = fd.assemble(ns, a, 0.0).tocsc()
        F = gpu_lib.rhif_factor(csrs[i], ns, 8, 1e-3, precision=precision)
        u1, it1, rr1 = F.pcg(fs[i], rtol=1e-10)
        if precision == "fp64":
            assert its[i] == it1
        else:
            assert all(abs(x - y) <= 1 for x, y in zip(its[i], it1))
        for r in range(3):
            assert rr[i][r] <= 1.5e-10
            ud = spla.spsolve(A, fs[i][r].cpu().numpy())
            assert np.linalg.norm(us[i][r].cpu().numpy() - ud) <= 1e-7 * np.linalg.norm(ud)
        F.free()
    # the same through rhif_pcg on concatenated vectors
    fc = torch.cat([f for f in fs], dim=1).contiguous()
    uc, itc, rrc = FB.pcg(fc, rtol=1e-10)
    assert itc == its
    for i, part in enumerate(FB.split(uc)):
        np.testing.assert_allclose(part.cpu().numpy(), us[i].cpu().numpy(), rtol=0,
                                   atol=1e-13 * float(us[i].abs().max()))
    FB.free()


def test_merged_batch_3d_matches_single_problems(gpu_lib):
    probs = _problems([15, (11, 9, 13), 7, 16], d=3, seed=500)
    FB, _, _ = _check_against_singles(gpu_lib, probs, 4, 1e-3, "fp64", b=1e-2, edge=True)
    FB.free()


def test_merged_batch_fp64_against_oracle(gpu_lib):
    probs = _problems([31, 63, 20], lohi=(1e-4, 1e4), seed=600)
    csrs = [gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0) for ns, a in probs]
    FB = gpu_lib.rhif_factor_batch(csrs, [ns for ns, _ in probs], 8, 1e-3, precision="fp64")
    xs = [np.random.default_rng(9 + i).standard_normal(int(np.prod(ns))) for i, (ns, _) in enumerate(probs)]
    Ax = []
    for i, (ns, a) in enumerate(probs):
        Ax.append(fd.assemble(ns, a, 0.0) @ xs[i])
    yb = FB.apply(_dev(np.concatenate(xs))).cpu().numpy()
    eb = FB.apply(_dev(np.concatenate(Ax))).cpu().numpy()
    for i, (ns, a) in enumerate(probs):
        A = fd.assemble(ns, a, 0.0)
        Fo = phif.factor(A, ns, 8, 1e-3)
        lo, hi = FB.dof_base[i], FB.dof_base[i + 1]
        yo = phif.solve(Fo, xs[i])
        assert np.linalg.norm(yb[lo:hi] - yo) <= 1e-9 * np.linalg.norm(yo)
        eo = np.linalg.norm(phif.solve(Fo, Ax[i]) - xs[i]) / np.linalg.norm(xs[i])
        eg = np.linalg.norm(eb[lo:hi] - xs[i]) / np.linalg.norm(xs[i])
        assert eg <= 2 * eo + 1e-12
    # the batch's A against the oracle's assembly
    ab = FB.spmv(_dev(np.concatenate(xs))).cpu().numpy()
    np.testing.assert_allclose(ab, np.concatenate(Ax), rtol=1e-13, atol=1e-13 * np.abs(ab).max())
    FB.free()


def test_merged_batch_rejects_mixed_dimensions(gpu_lib):
    p2 = _problems([15])[0]
    p3 = _problems([7], d=3)[0]
    csrs = [gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0) for ns, a in (p2, p3)]
    with pytest.raises(gpu_lib.RhifError) as e:
        gpu_lib.rhif_factor_batch(csrs, [p2[0], p3[0]], 4, 1e-3)
    assert e.value.code == -1


def test_batch_device_pcg_loop_matches_host_loop(gpu_lib):
    """rhif_pcg_batch runs its iterations on the device (one CUDA graph whose
    conditional loop tests every (problem, right-hand side) pair there); with
    per-launch timing on it runs them from the host.  Both give the same
    solutions bit for bit and the same per-pair iteration counts, also when
    maxit stops them (NOT_CONVERGED)."""
    probs = _problems([23, 31, (17, 29)], seed=410)
    csrs = [gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0) for ns, a in probs]
    FB = gpu_lib.rhif_factor_batch(csrs, [ns for ns, _ in probs], 4, 1e-3, precision="fp32")
    rng = np.random.default_rng(23)
    fs = [_dev(rng.standard_normal((2, int(np.prod(ns))))) for ns, _ in probs]
    for rtol, maxit, check in ((1e-11, 1000, True), (1e-14, 2, False)):
        ud, itd, _ = FB.pcg_batch(fs, rtol=rtol, maxit=maxit, check=check)
        try:
            gpu_lib.rhif_set_timing(True)
            uh, ith, _ = FB.pcg_batch(fs, rtol=rtol, maxit=maxit, check=check)
        finally:
            gpu_lib.rhif_set_timing(False)
        assert itd == ith
        for a, b in zip(ud, uh):
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        if maxit == 2:
            assert all(i == [2, 2] for i in itd)
    FB.free()
