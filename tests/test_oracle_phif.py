"""Pins for the oracle's PHIF factorization and application (Secs. 2-4).

The strongest pins rebuild the paper's operators as explicit dense N x N
matrices on tiny grids -- the elimination matrix of Eq. (2.1), the
preconditioning matrix of Eq. (2.3), the zeroing matrix of Eq. (2.2) and the
elimination of the redundant DOFs -- straight from the level snapshots and the
geometric grouping, and check that they reproduce the oracle's next-level
matrices and its F^{-1} (Eqs. 3.1-3.3).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import dense, fd, phif, tree


def _problem(ns, lo=1e-2, hi=1e2, b=0.0, seed=11):
    a = W.log_uniform_pixels(ns, lo, hi, seed)
    return fd.assemble(ns, a, b)


def _full(S):
    """Sparse snapshot (zero rows on eliminated DOFs) -> paper's matrix with
    identity on the eliminated DOFs."""
    M = S.toarray()
    dead = np.diag(M) == 0.0
    M[dead, dead] = 1.0
    return M, ~dead


def _explicit_level(ns, leaf, lvl, snap, level_rec, precondition=True):
    """Explicit E_l, C_l and K_l (as lists of factors) from a level snapshot."""
    width = leaf << lvl
    A0, act0 = _full(snap["A"])
    N = A0.shape[0]
    # E_l = prod over cells of Eq. (2.1); the row blocks of distinct cells never overlap
    E = np.eye(N)
    cells = [g for g in tree.groups(ns, np.nonzero(act0)[0], width) if g[1] == 0]
    for _, _, I in cells:
        rest = np.setdiff1d(np.arange(N), I)
        Lc = np.linalg.cholesky(A0[np.ix_(I, I)])
        E[np.ix_(I, I)] = np.linalg.inv(Lc).T
        E[np.ix_(I, rest)] = -np.linalg.solve(A0[np.ix_(I, I)], A0[np.ix_(rest, I)].T)
    A1, act1 = _full(snap["A1"])
    # C_l = block diag of L_g^{-T} over the separator groups, Eq. (2.3); the
    # diagonal local preconditioner uses diag(A_gg)^{-1/2} instead
    C = np.eye(N)
    if precondition:
        for _, _, g in tree.groups(ns, np.nonzero(act1)[0], width):
            C[np.ix_(g, g)] = _local_precond(A1[np.ix_(g, g)], precondition)
    return E, C, A0, A1


def _local_precond(Agg, mode):
    if mode == "diag":
        return np.diag(1.0 / np.sqrt(np.diag(Agg)))
    return np.linalg.inv(np.linalg.cholesky(Agg)).T


def _explicit_skeletonization(A2, units):
    """Apply Z_I E_Ir unit by unit (Sec. 2.2) to A2 after replacing A_{R,Ir} by
    A_{R,Is} T; returns (K, result, size of the replaced perturbation)."""
    N = A2.shape[0]
    M = A2.copy()
    K = np.eye(N)
    pert = 0.0
    for u in units:
        if u.rd.size == 0:
            continue
        R = np.setdiff1d(np.arange(N), u.e)
        new = M[np.ix_(R, u.sk)] @ u.T
        pert = max(pert, np.abs(new - M[np.ix_(R, u.rd)]).max())
        M[np.ix_(R, u.rd)] = new
        M[np.ix_(u.rd, R)] = new.T
        Z = np.eye(N)
        Z[np.ix_(u.sk, u.rd)] = -u.T
        M = Z.T @ M @ Z
        rest = np.setdiff1d(np.arange(N), u.rd)
        Arr = M[np.ix_(u.rd, u.rd)]
        Er = np.eye(N)
        Er[np.ix_(u.rd, u.rd)] = np.linalg.inv(np.linalg.cholesky(Arr)).T
        Er[np.ix_(u.rd, rest)] = -np.linalg.solve(Arr, M[np.ix_(rest, u.rd)].T)
        M = Er.T @ M @ Er
        K = K @ Z @ Er
    return K, M, pert


@pytest.mark.parametrize("ns,leaf,tol,edge_skel,precond", [
    ((15, 15), 4, 1e-4, False, True),
    ((13, 13), 4, 1e-3, False, True),     # padded tree
    ((15, 15), 4, 1e-4, False, False),    # plain HIF
    ((7, 7, 7), 4, 1e-3, True, True),     # 3D, faces then edges (Remark 3.1)
    ((11, 11, 11), 4, 1e-3, False, True),  # 3D padded, two levels
    ((15, 15), 4, 1e-4, False, "diag"),   # diagonal local preconditioner
    ((7, 7, 7), 4, 1e-3, True, "diag"),
])
def test_explicit_operator_products(ns, leaf, tol, edge_skel, precond):
    A = _problem(ns, b=0.01 if len(ns) == 3 else 0.0)
    F = phif.factor(A, ns, leaf, tol, precondition=precond, edge_skel=edge_skel, snapshots=True)
    N = A.shape[0]
    Rs = []
    for lvl, (snap, lv) in enumerate(zip(F.snapshots, F.levels)):
        E, C, A0, A1 = _explicit_level(ns, leaf, lvl, snap, lv, precond)
        scale = np.abs(A0).max()
        np.testing.assert_allclose(E.T @ A0 @ E, A1, atol=1e-12 * scale)
        A2, act2 = _full(snap["A2"])
        np.testing.assert_allclose(C.T @ A1 @ C, A2, atol=1e-12 * np.abs(A1).max())
        if precond == "diag":   # unit diagonal
            for _, _, g in tree.groups(ns, np.nonzero(act2)[0], leaf << lvl):
                np.testing.assert_allclose(np.diag(A2[np.ix_(g, g)]), np.ones(g.size), atol=1e-12)
        elif precond:   # unit block diagonal (Sec. 2.3)
            for _, _, g in tree.groups(ns, np.nonzero(act2)[0], leaf << lvl):
                np.testing.assert_allclose(A2[np.ix_(g, g)], np.eye(g.size), atol=1e-12)
        Ktot = np.eye(N)
        M = A2
        for pi, ph in enumerate(lv.phases):
            if pi == 1:   # second pass: precondition edges and corners again
                Mf = M.copy()
                C2 = np.eye(N)
                for g in ph.groups:
                    C2[np.ix_(g.g, g.g)] = _local_precond(Mf[np.ix_(g.g, g.g)], precond)
                M = C2.T @ Mf @ C2
                Ktot = Ktot @ C2
            K, M, pert = _explicit_skeletonization(M, ph.units)
            assert pert <= 50 * tol * np.abs(A2).max()
            Ktot = Ktot @ K
        A3, _ = _full(snap["A3"])
        np.testing.assert_allclose(M, A3, atol=1e-11 * np.abs(A2).max())
        Rs.append(E @ C @ Ktot)
    # F^{-1} = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T  (Eq. 3.2)
    AL = np.eye(N)
    AL[np.ix_(F.S, F.S)] = F.BL @ F.BL.T
    P = np.eye(N)
    for R in Rs:
        P = P @ R
    Finv = P @ np.linalg.solve(AL, P.T)
    x = np.random.default_rng(0).standard_normal(N)
    y = phif.solve(F, x)
    np.testing.assert_allclose(y, Finv @ x, rtol=0, atol=1e-9 * np.abs(Finv @ x).max())
    # F = R_0^{-T} ... A_L ... R_0^{-1}  (Eq. 3.1)
    Fm = np.linalg.solve(P.T, np.linalg.solve(P.T, AL.T).T).T
    np.testing.assert_allclose(phif.matvec(F, x), Fm @ x, atol=1e-9 * np.abs(Fm @ x).max())


def test_skeleton_block_form_after_preconditioning():
    """Sec. 3.3: after preconditioning, Z^T A Z on a unit is [[I+T^T T, -T^T], [-T, I]]."""
    ns = (31, 31)
    A = _problem(ns, 1e-3, 1e3)
    F = phif.factor(A, ns, 8, 1e-4, snapshots=True)
    for snap, lv in zip(F.snapshots, F.levels):
        A2, _ = _full(snap["A2"])
        for u in lv.phases[0].units:
            if u.rd.size == 0:
                continue
            order = np.concatenate([u.rd, u.sk])
            k, r = u.sk.size, u.rd.size
            Z = np.eye(r + k)
            Z[r:, :r] = -u.T
            blk = Z.T @ A2[np.ix_(order, order)] @ Z
            want = np.block([[np.eye(r) + u.T.T @ u.T, -u.T.T], [-u.T, np.eye(k)]])
            np.testing.assert_allclose(blk, want, atol=1e-11)


@pytest.mark.parametrize("ns,leaf,edge_skel,precond", [
    ((7, 7), 4, False, True), ((15, 15), 4, False, True), ((31, 31), 8, False, True),
    ((20, 23), 4, False, True), ((7, 7, 7), 4, False, True), ((15, 15, 15), 4, True, True),
    ((9, 6, 7), 4, False, True), ((20, 23), 4, False, "diag"), ((7, 7, 7), 4, True, "diag"),
])
def test_tol_zero_is_exact(ns, leaf, edge_skel, precond):
    """tol = 0: nothing is dropped, F = A and F^{-1} A = I to roundoff."""
    A = _problem(ns, b=0.01)
    F = phif.factor(A, ns, leaf, 0.0, edge_skel=edge_skel, precondition=precond)
    x = np.random.default_rng(1).standard_normal(A.shape[0])
    np.testing.assert_allclose(phif.matvec(F, x), A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())
    y = phif.solve(F, A @ x)
    assert np.linalg.norm(y - x) <= 1e-10 * np.linalg.norm(x)
    u, it, rr = phif.pcg(A, x, M=lambda r: phif.solve(F, r), rtol=1e-12)
    assert it == 1 and rr < 1e-12
    u_direct = spla.spsolve(A.tocsc(), x)
    assert np.linalg.norm(u - u_direct) <= 1e-10 * np.linalg.norm(u_direct)


def test_sine_modes_are_reproduced_by_the_exact_factor():
    """a = 1: F^{-1} v_jk = v_jk / lambda_jk with the closed-form eigenvalues."""
    ns = (31, 31)
    A = fd.assemble(ns, np.ones(W.pixel_shape(ns)), 0.0)
    F = phif.factor(A, ns, 8, 0.0)
    h = 1.0 / 32
    xs = np.arange(1, 32) * h
    X, Y = np.meshgrid(xs, xs)   # Y rows, X cols -> x fastest after ravel
    for j, k in [(1, 1), (3, 17), (31, 2), (16, 16)]:
        v = (np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)).ravel()
        lam = 4 / h ** 2 * (np.sin(j * np.pi * h / 2) ** 2 + np.sin(k * np.pi * h / 2) ** 2)
        np.testing.assert_allclose(phif.solve(F, v), v / lam, atol=1e-12 / lam)


def test_sine_spectrum_of_preconditioned_laplacian_within_solve_error():
    ns = (31, 31)
    A = fd.assemble(ns, np.ones(W.pixel_shape(ns)), 0.0)
    F = phif.factor(A, ns, 4, 1e-3)
    es = phif.solve_error(A, F, seed=3)
    h = 1.0 / 32
    xs = np.arange(1, 32) * h
    X, Y = np.meshgrid(xs, xs)
    for j, k in [(1, 1), (2, 5), (30, 30), (9, 21)]:
        v = (np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)).ravel()
        lam = 4 / h ** 2 * (np.sin(j * np.pi * h / 2) ** 2 + np.sin(k * np.pi * h / 2) ** 2)
        q = lam * (v @ v) / (v @ phif.matvec(F, v))   # generalized Rayleigh quotient v^T A v / v^T F v
        assert abs(q - 1.0) <= 2 * es + 1e-12


def test_symmetry_and_cell_order_independence():
    ns = (31, 31)
    A = _problem(ns, 1e-3, 1e3)
    F1 = phif.factor(A, ns, 4, 1e-4)
    rng = np.random.default_rng(4)
    F2 = phif.factor(A, ns, 4, 1e-4, cell_order=lambda lvl, n: rng.permutation(n))
    x, y = rng.standard_normal((2, A.shape[0]))
    a1, a2 = x @ phif.solve(F1, y), y @ phif.solve(F1, x)
    assert abs(a1 - a2) <= 1e-12 * abs(a1)
    assert F1.ranks == F2.ranks
    np.testing.assert_allclose(phif.solve(F2, x), phif.solve(F1, x), rtol=0,
                               atol=1e-11 * np.abs(phif.solve(F1, x)).max())


def test_apply_error_scales_with_tolerance():
    ns = (63, 63)
    A = _problem(ns, 1e-2, 1e2)
    prev = None
    for tol in [1e-3, 1e-6, 1e-9]:
        F = phif.factor(A, ns, 8, tol)
        ea = phif.apply_error(A, F, seed=5)
        assert ea <= 30 * tol
        if prev is not None:
            assert ea < prev
        prev = ea


def test_preconditioning_reduces_solve_error_on_high_contrast_field():
    """Sec. 4 headline: PHIF e_s well below HIF e_s at the same tolerance."""
    ns = (63, 63)
    a = W.paper_quantized_field(ns, seed=9)
    A = fd.assemble(ns, a, 0.0)
    Fp = phif.factor(A, ns, 8, 1e-6, precondition=True)
    Fh = phif.factor(A, ns, 8, 1e-6, precondition=False)
    es_p = phif.solve_error(A, Fp, seed=1)
    es_h = phif.solve_error(A, Fh, seed=1)
    assert es_p * 10 < es_h
    _, it_p, _ = phif.pcg(A, np.ones(A.shape[0]), M=lambda r: phif.solve(Fp, r), rtol=1e-12)
    _, it_h, _ = phif.pcg(A, np.ones(A.shape[0]), M=lambda r: phif.solve(Fh, r), rtol=1e-12)
    assert it_p <= it_h
    # the diagonal local preconditioner (concluding section) lies in between:
    # it rescales every separator group to unit diagonal, which removes part of
    # the coefficient contrast the IDs see (about 5x smaller e_s than HIF here)
    Fd = phif.factor(A, ns, 8, 1e-6, precondition="diag")
    es_d = phif.solve_error(A, Fd, seed=1)
    assert es_d * 2 < es_h and es_p <= es_d


def test_pcg_with_factor_on_small_benchmark_grid():
    p = W.config_problem(0)
    A = fd.assemble(p.ns, p.a, p.b)
    F = phif.factor(A, p.ns, p.leaf, p.tol)
    u, it, rr = phif.pcg(A, p.f, M=lambda r: phif.solve(F, r), rtol=1e-12)
    assert rr < 1e-11 and it < 30
    assert [len(r) for r in F.ranks] == [480, 112, 24, 4]   # interior edges per level


def test_not_spd_is_reported():
    ns = (15, 15)
    A = _problem(ns).tolil()
    A[37, 37] = -1.0
    with pytest.raises(dense.NotSPD):
        phif.factor(A.tocsr(), ns, 4, 1e-3)


@pytest.mark.parametrize("ns,leaf,tol", [((15, 15), 4, 1e-2), ((15, 15), 4, 1e-4), ((7, 7, 7), 4, 1e-2)])
def test_power_norm_against_dense_two_norm(ns, leaf, tol):
    """Sec. 4 estimators pinned to the dense 2-norm (singular value routine):
    M_s = I - A F^{-1} and M_a = A - F are formed column by column.  The power
    iteration on M^T M can only underestimate ||M||_2 (sqrt ||M^T M v|| <=
    ||M||_2 for a unit v), reaches it to 1e-6 when run to a 1e-13 change (the
    slowest case has nearly equal top singular values), and with the paper's
    1e-2 stopping rule lands at most 15% below it (13% seen); e_a, a ratio of
    two such estimates, lands within 15% (10% seen)."""
    a = W.log_uniform_pixels(ns, 1e-2, 1e2, seed=21)
    A = fd.assemble(ns, a, 0.0)
    N = A.shape[0]
    F = phif.factor(A, ns, leaf, tol)
    I = np.eye(N)
    Ad = A.toarray()
    Ms = I - Ad @ np.column_stack([phif.solve(F, I[:, j]) for j in range(N)])
    Ma = Ad - np.column_stack([phif.matvec(F, I[:, j]) for j in range(N)])
    for M in (Ms, Ma, Ad):
        true = np.linalg.norm(M, 2)
        tight = phif.power_norm(lambda v: M @ v, lambda v: M.T @ v, N, seed=0, rel=1e-13, maxit=50000)
        assert abs(tight / true - 1.0) <= 1e-6
        for seed in range(4):
            est = phif.power_norm(lambda v: M @ v, lambda v: M.T @ v, N, seed=seed)
            assert est <= true * (1 + 1e-12)
            assert est >= 0.85 * true
    es_true = np.linalg.norm(Ms, 2)
    ea_true = np.linalg.norm(Ma, 2) / np.linalg.norm(Ad, 2)
    for seed in range(4):
        assert 0.85 * es_true <= phif.solve_error(A, F, seed=seed) <= es_true * (1 + 1e-12)
        assert abs(phif.apply_error(A, F, seed=seed) / ea_true - 1.0) <= 0.15
