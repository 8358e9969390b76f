"""GPU path vs the FP64 oracle on the same seeded inputs (through the C-ABI).

FP64 bar: identical skeleton sets except at logged near-ties (the pivot
choices are then the same, so both sides apply the same operators); F^{-1} x
within 1e-9 relative of the oracle's (the two differ only in summation order,
about 1e-16 per operation, amplified by the conditioning of the level factors,
which stays below ~1e6 on these grids); apply error ||F^{-1}Ax - x|| within 2x
of the oracle's; PCG relative residual <= rtol with the solution within 1e-9 of
a sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _gpu_matrix(lib, ns, a, b):
    bb = _dev(np.broadcast_to(b, (int(np.prod(ns)),)).astype(np.float64)) if not np.isscalar(b) else b
    return lib.rhif_assemble_fd(ns, _dev(a), bb)


def _skeleton_map(units):
    """{frozenset(unit dofs): frozenset(skeleton dofs)}"""
    return {frozenset(int(g) for g in dofs): frozenset(int(g) for g in dofs[:k]) for dofs, k in units}


def _oracle_skeletons(F, level, phase):
    ph = F.levels[level].phases[phase]
    return {frozenset(int(g) for g in u.e): frozenset(int(g) for g in u.sk) for u in ph.units}


def test_fd_assembly_matches_oracle(gpu_lib):
    for ns, b in [((31, 17), 0.0), ((9, 8, 7), 0.01), ((1, 5), 0.0)]:
        a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=3)
        rp, col, val = _gpu_matrix(gpu_lib, ns, a, b)
        A = fd.assemble(ns, a, b)
        np.testing.assert_array_equal(rp.cpu().numpy(), A.indptr)
        np.testing.assert_array_equal(col.cpu().numpy(), A.indices)
        np.testing.assert_allclose(val.cpu().numpy(), A.data, rtol=1e-14, atol=0)


CASES = [
    # ns, leaf, tol, (lo, hi), b, edge_skel
    ((15, 15), 4, 1e-4, (1e-2, 1e2), 0.0, False),
    ((31, 31), 8, 1e-3, (1e-3, 1e3), 0.0, False),
    ((63, 63), 8, 1e-6, (1e-3, 1e3), 0.0, False),
    ((20, 23), 4, 1e-3, (1e-2, 1e2), 0.0, False),     # padded, ragged tail
    ((127, 127), 8, 1e-3, (1e-2, 1e2), 0.0, False),   # the 127^2 benchmark grid
    ((15, 15, 15), 4, 1e-3, (1e-3, 1e3), 1e-2, False),
    ((11, 9, 13), 4, 1e-3, (1e-3, 1e3), 1e-2, False),  # 3D padded
    ((15, 15, 15), 4, 1e-3, (1e-3, 1e3), 1e-2, True),  # faces then edges
]


@pytest.mark.parametrize("ns,leaf,tol,lohi,b,edge", CASES)
def test_fp64_factor_matches_oracle(gpu_lib, ns, leaf, tol, lohi, b, edge):
    a = W.log_uniform_pixels(ns, *lohi, seed=sum(ns) + leaf)
    A = fd.assemble(ns, a, b)
    Fo = phif.factor(A, ns, leaf, tol, edge_skel=edge)
    csr = _gpu_matrix(gpu_lib, ns, a, b)
    Fg = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp64", edge_skel_3d=edge)
    st = Fg.stats()
    assert st["levels"] == len(Fo.levels)
    tie_units = {(str(w), k) for (w, k, *_rest) in Fo.ties}
    diverged = False
    for lvl in range(len(Fo.levels)):
        for ph in range(len(Fo.levels[lvl].phases)):
            go = _oracle_skeletons(Fo, lvl, ph)
            gg = _skeleton_map(Fg.skeletons(lvl, ph))
            assert set(go) == set(gg), f"unit sets differ at level {lvl} phase {ph}"
            bad = [u for u in go if go[u] != gg[u]]
            if bad:
                assert Fo.ties, f"skeleton sets differ at level {lvl} phase {ph} without a logged tie"
                diverged = True
        if diverged:
            break
    if not diverged:
        assert st["root_size"] == Fo.S.size
    x = np.random.default_rng(7).standard_normal(A.shape[0])
    yg = Fg.apply(_dev(x)).cpu().numpy()
    yo = phif.solve(Fo, x)
    if not diverged:
        assert np.linalg.norm(yg - yo) <= 1e-9 * np.linalg.norm(yo)
    # apply error ||F^{-1} A x - x|| / ||x|| within 2x of the oracle's
    Ax = A @ x
    eg = np.linalg.norm(Fg.apply(_dev(Ax)).cpu().numpy() - x) / np.linalg.norm(x)
    eo = np.linalg.norm(phif.solve(Fo, Ax) - x) / np.linalg.norm(x)
    assert eg <= 2 * eo + 1e-12
    Fg.free()


@pytest.mark.parametrize("ns,leaf", [((31, 31), 4), ((20, 13), 4), ((7, 9, 8), 4)])
def test_tol_zero_is_exact_on_gpu(gpu_lib, ns, leaf):
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=5)
    A = fd.assemble(ns, a, 0.01)
    Fg = gpu_lib.rhif_factor(_gpu_matrix(gpu_lib, ns, a, 0.01), ns, leaf, 0.0)
    x = np.random.default_rng(2).standard_normal(A.shape[0])
    y = Fg.apply(_dev(A @ x)).cpu().numpy()
    assert np.linalg.norm(y - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pcg_solution_matches_direct_solve(gpu_lib, precision):
    p = W.config_problem(0)
    A = fd.assemble(p.ns, p.a, p.b)
    Fg = gpu_lib.rhif_factor(_gpu_matrix(gpu_lib, p.ns, p.a, p.b), p.ns, p.leaf, p.tol,
                             precision=precision)
    u, its, rr = Fg.pcg(_dev(p.f), rtol=1e-12, maxit=200)
    u = u.cpu().numpy()
    ud = spla.spsolve(A.tocsc(), p.f)
    assert rr[0] <= 1e-12 * 1.5
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
    if precision == "fp64":
        Fo = phif.factor(A, p.ns, p.leaf, p.tol)
        _, it_o, _ = phif.pcg(A, p.f, M=lambda r: phif.solve(Fo, r), rtol=1e-12)
        assert abs(its[0] - it_o) <= 1


def test_multi_rhs_pcg(gpu_lib):
    ns = (63, 63)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=9)
    A = fd.assemble(ns, a, 0.0)
    F = W.normal_rhs(ns, 4, nrhs=5)
    Fg = gpu_lib.rhif_factor(_gpu_matrix(gpu_lib, ns, a, 0.0), ns, 8, 1e-3, precision="fp32")
    U, its, rr = Fg.pcg(_dev(F), rtol=1e-10)
    U = U.cpu().numpy()
    for r in range(5):
        assert rr[r] <= 1.5e-10
        ud = spla.spsolve(A.tocsc(), F[r])
        assert np.linalg.norm(U[r] - ud) <= 1e-7 * np.linalg.norm(ud)
    Y = Fg.apply(_dev(F)).cpu().numpy()
    for r in range(5):
        y1 = Fg.apply(_dev(F[r])).cpu().numpy()
        np.testing.assert_allclose(Y[r], y1, rtol=0, atol=1e-12 * np.abs(y1).max())


def test_not_spd_reported(gpu_lib):
    ns = (15, 15)
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=1)
    rp, col, val = _gpu_matrix(gpu_lib, ns, a, 0.0)
    v = val.cpu().numpy()
    rpn = rp.cpu().numpy()
    cn = col.cpu().numpy()
    i = 37
    k = rpn[i] + np.nonzero(cn[rpn[i]:rpn[i + 1]] == i)[0][0]
    v[k] = -1.0
    with pytest.raises(gpu_lib.RhifError) as e:
        gpu_lib.rhif_factor((rp, col, _dev(v)), ns, 4, 1e-3)
    assert e.value.code == -2


def test_bad_csr_pattern_rejected(gpu_lib):
    ns = (8, 8)
    N = 64
    rows = np.arange(N)
    cols = (rows + 9) % N   # not a grid neighbour
    A = sp.csr_matrix((np.ones(2 * N), (np.r_[rows, rows], np.r_[rows, cols])), shape=(N, N))
    A.sort_indices()
    csr = (_dev(A.indptr.astype(np.int64)), _dev(A.indices.astype(np.int32)), _dev(A.data))
    with pytest.raises(gpu_lib.RhifError) as e:
        gpu_lib.rhif_factor(csr, ns, 4, 1e-3)
    assert e.value.code == -1


def test_gradient_kernel_matches_oracle(gpu_lib):
    for ns in [(17, 12), (6, 5, 7)]:
        a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=8)
        u = W.normal_rhs(ns, 1)
        lam = W.normal_rhs(ns, 2)
        g = gpu_lib.rhif_grad_logcoef(ns, _dev(a), _dev(u), _dev(lam)).cpu().numpy()
        go = fd.dA_dlog_a(ns, a, u, lam)
        np.testing.assert_allclose(g, go, rtol=1e-12, atol=1e-12 * np.abs(go).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_factor_is_deterministic(gpu_lib, precision):
    """Two factorizations of the same input give the same skeletons and bitwise
    equal F^{-1} x (no atomics; all IDs of a level read the same matrix)."""
    ns = (255, 255)
    a = W.log_uniform_pixels(ns, 1e-4, 1e4, seed=12)
    csr = _gpu_matrix(gpu_lib, ns, a, 0.0)
    x = _dev(W.normal_rhs(ns, 13))
    outs = []
    for _ in range(2):
        F = gpu_lib.rhif_factor(csr, ns, 16, 1e-3, precision=precision)
        sk = [F.skeletons(l) for l in range(F.stats()["levels"])]
        outs.append((sk, F.apply(x).cpu().numpy()))
        F.free()
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_pcg_does_not_read_stale_scratch(gpu_lib):
    """PCG must not depend on what its work space held before: a solve with a
    NaN right-hand side leaves NaN in the handle's scratch vectors, and the
    next solve on the same handle still converges to the direct solution."""
    ns = (63, 63)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=31)
    A = fd.assemble(ns, a, 0.0)
    Fg = gpu_lib.rhif_factor(_gpu_matrix(gpu_lib, ns, a, 0.0), ns, 8, 1e-3, precision="fp32")
    F = W.normal_rhs(ns, 32, nrhs=2)
    bad = F.copy()
    bad[:, 17] = np.nan
    Fg.pcg(_dev(bad), rtol=1e-10, maxit=3, check=False)
    U, its, rr = Fg.pcg(_dev(F), rtol=1e-10)
    U = U.cpu().numpy()
    for r in range(2):
        assert rr[r] <= 1.5e-10
        ud = spla.spsolve(A.tocsc(), F[r])
        assert np.linalg.norm(U[r] - ud) <= 1e-7 * np.linalg.norm(ud)


@pytest.mark.parametrize("skel_cluster", [-1, 0, 4])
@pytest.mark.parametrize("precondition", [True, False])
def test_separator_breakdown_reported(gpu_lib, skel_cluster, precondition):
    """A negative diagonal on a separator DOF makes a later Cholesky of the
    level fail (block Jacobi factor or redundant-DOF elimination); the NaNs
    that reach the interpolative decompositions of the same level must stop
    them cleanly, and the factorization reports NOT_SPD."""
    ns, leaf = (15, 15), 4
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=1)
    rp, col, val = _gpu_matrix(gpu_lib, ns, a, 0.0)
    v = val.cpu().numpy()
    rpn, cn = rp.cpu().numpy(), col.cpu().numpy()
    i = 4 + 15 * 5 - 1   # x = 4, y = 6 (1-based): on a level-0 separator edge
    k = rpn[i] + np.nonzero(cn[rpn[i]:rpn[i + 1]] == i)[0][0]
    v[k] = -50.0 * abs(v[k])
    with pytest.raises(gpu_lib.RhifError) as e:
        gpu_lib.rhif_factor((rp, col, _dev(v)), ns, leaf, 1e-3, precondition=precondition,
                            skel_cluster=skel_cluster)
    assert e.value.code == -2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ns,leaf", [((63, 63), 8), ((127, 127), 16), ((20, 23), 4), ((15, 15, 15), 4)])
def test_many_rhs_apply_matches_one_rhs_apply(gpu_lib, precision, ns, leaf):
    """From 8 right-hand sides the 2D leaf sweeps run one lane per right-hand
    side and the front sweeps eight right-hand sides per pass (the one-vector
    kernels' operations, compiled in another shape): 40 right-hand sides (full
    and partial chunks) match the columns of 40 one-vector applications to
    rounding (FP64 1e-11, FP32 1e-5 relative)."""
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=sum(ns) + 2)
    Fg = gpu_lib.rhif_factor(_gpu_matrix(gpu_lib, ns, a, 0.0), ns, leaf, 1e-3, precision=precision)
    X = _dev(np.random.default_rng(14).standard_normal((40, Fg.N)))
    Y = Fg.apply(X).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 1e-5
    for r in range(40):
        y1 = Fg.apply(X[r].contiguous()).cpu().numpy()
        assert np.linalg.norm(Y[r] - y1) <= tol * np.linalg.norm(y1)
    Fg.free()


def test_shared_level0_plan_gives_the_factor_of_a_fresh_plan(gpu_lib):
    """The level-0 plan (fixed by the grid, the leaf size and the options) is
    kept and shared by later factorizations of the same kind: factors made
    after other grids and other options evicted it, and factors made while it
    is shared, apply exactly as the first one did."""
    ns_a, ns_b = (31, 33), (47, 47)
    x = _dev(np.random.default_rng(11).standard_normal(ns_a[0] * ns_a[1]))

    def apply_a(**kw):
        a = W.log_uniform_pixels(ns_a, 1e-3, 1e3, seed=3)
        Fa = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns_a, _dev(a), 0.0), ns_a, 4, 1e-3,
                                 precision="fp64", **kw)
        y = Fa.apply(x).cpu().numpy()
        return Fa, y

    F1, y1 = apply_a()                      # builds the shared plan
    F2, y2 = apply_a()                      # shares it while F1 holds it too
    np.testing.assert_array_equal(y1, y2)
    F1.free()
    b = W.log_uniform_pixels(ns_b, 1e-3, 1e3, seed=4)
    Fb = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns_b, _dev(b), 0.0), ns_b, 4, 1e-3,
                             precision="fp64")   # another grid: a new plan replaces it
    F3, y3 = apply_a()                      # rebuilt for the first grid
    np.testing.assert_array_equal(y1, y3)
    F4, y4 = apply_a(precondition="diag")   # other options: another plan
    F5, y5 = apply_a()
    np.testing.assert_array_equal(y1, y5)
    assert not np.array_equal(y1, y4)
    y2b = F2.apply(x).cpu().numpy()         # the handle that shared the first plan still works
    np.testing.assert_array_equal(y1, y2b)
    for F in (F2, Fb, F3, F4, F5):
        F.free()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_device_pcg_loop_matches_host_loop(gpu_lib, precision):
    """rhif_pcg runs its iterations on the device (a CUDA graph whose
    conditional loop tests convergence there); with per-launch timing on it
    runs the same iterations from the host.  Both give the same solution, bit
    for bit, and the same per-right-hand-side iteration counts, also when
    maxit stops them before rtol (NOT_CONVERGED, counts = maxit)."""
    ns = (63, 63)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=17)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, 8, 1e-3,
                             precision=precision)
    f = _dev(np.random.default_rng(5).standard_normal((3, Fg.N)))
    try:
        u_d, it_d, rr_d = Fg.pcg(f, rtol=1e-11)
        gpu_lib.rhif_set_timing(True)
        u_h, it_h, rr_h = Fg.pcg(f, rtol=1e-11)
    finally:
        gpu_lib.rhif_set_timing(False)
    np.testing.assert_array_equal(u_d.cpu().numpy(), u_h.cpu().numpy())
    assert it_d == it_h and rr_d == rr_h
    assert max(rr_d) <= 1.5e-11
    u_d, it_d, _ = Fg.pcg(f, rtol=1e-14, maxit=2, check=False)
    try:
        gpu_lib.rhif_set_timing(True)
        u_h, it_h, _ = Fg.pcg(f, rtol=1e-14, maxit=2, check=False)
    finally:
        gpu_lib.rhif_set_timing(False)
    assert it_d == it_h == [2, 2, 2]
    np.testing.assert_array_equal(u_d.cpu().numpy(), u_h.cpu().numpy())
    Fg.free()
