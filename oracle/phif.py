"""PHIF factorization, application and PCG (Sec. 3 and Sec. 4), plain FP64.

The active matrix ``A_l`` is one global scipy.sparse matrix.  Each level
``l = 0..L-1`` applies, in the paper's order (Sec. 3.1 steps 1-3; Sec. 3.2
steps 1-3 and, when asked, Remark 3.1 steps 4-5):

1. cell elimination ``A_l' = E_l^T A_l E_l`` (Sec. 2.1, Eq. 2.1): for every
   cell interior ``I``, ``A_II = L L^T``, ``X = L^{-1} A_BI^T``,
   ``A_BB <- A_BB - X^T X``; ``B`` is every active DOF outside ``I`` with a
   nonzero entry in ``A[:, I]`` (so ``A_RI = 0`` for the rest);
2. block Jacobi preconditioning ``A_l'' = C_l^T A_l' C_l`` (Sec. 2.3,
   Eq. 2.3) over all separator groups (edges+corners in 2D;
   faces+edges+corners in 3D); skipped for plain HIF;
3. skeletonization ``A_{l+1} ~= K_l^T A_l'' K_l`` (Sec. 2.2, Eq. 2.2) of every
   edge (2D) / face (3D) group: ID of ``A_{R,I}`` with ``R`` = every other
   active DOF with a nonzero entry in ``A[:, I]``; zeroing ``Z_I`` with
   ``A_{R,Ir}`` dropped; elimination of the redundant DOFs ``Ir``.  All IDs of
   a level are computed from ``A_l''`` before any zeroing (the parallel order
   of Sec. 2.2).

After the last level the active block is factored densely, ``A_L = B_L B_L^T``
(Eq. 3.3), and ``F^{-1} = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T`` with
``R_l = E_l C_l K_l`` (Eq. 3.2).

Parity: pinned in the tests by exactness at ``tol = 0`` (F = A), by the
explicit dense operator products of Eqs. (2.1)-(2.3) on tiny grids, by the
unit block diagonal after preconditioning (Sec. 2.3), by the skeleton block
form ``[[I + T^T T, -T^T], [-T, I]]`` (Sec. 3.3), by symmetry and by cell-order
independence (Sec. 2.1); PCG (Sec. 4) by one-step convergence with the tol = 0
factor, finite termination on right-hand sides made of a few sine modes and the
classical CG iteration bound on the Laplacian.  The 3D edge skeletonization (Remark 3.1, which the
paper did not run) is "parity unpinned" as a reading; its implementation is
checked by the tol = 0 exactness test and the explicit operator products of
its second pass.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp

from . import tree
from .dense import NotSPD, cholesky, lsolve, ltsolve, interp_decomp


@dataclasses.dataclass
class CellRec:
    I: np.ndarray     # interior gids
    B: np.ndarray     # coupled boundary gids
    L: np.ndarray     # chol(A_II)
    X: np.ndarray     # L^{-1} A_BI^T, |I| x |B|


@dataclasses.dataclass
class GroupRec:
    g: np.ndarray     # gids
    L: np.ndarray     # chol(A_gg)


@dataclasses.dataclass
class SkelRec:
    e: np.ndarray     # gids of the unit, ascending
    sk: np.ndarray    # skeleton gids (pivot order)
    rd: np.ndarray    # redundant gids (pivot order)
    T: np.ndarray     # k x |rd|, A_{R,rd} ~= A_{R,sk} T
    L: np.ndarray     # chol of the zeroed redundant block
    X: np.ndarray     # L^{-1} Atilde_{sk,rd}^T, |rd| x k
    key: tuple = ()


@dataclasses.dataclass
class Phase:
    """One preconditioning + skeletonization pass inside a level."""
    groups: list
    units: list


@dataclasses.dataclass
class Level:
    cells: list
    phases: list
    active_after: int = 0


@dataclasses.dataclass
class Factor:
    N: int
    ns: tuple
    leaf: int
    tol: float
    precondition: bool
    levels: list
    S: np.ndarray         # root active gids
    BL: np.ndarray        # chol(A_L)
    ties: list
    snapshots: list | None = None

    @property
    def ranks(self):
        return [[u.sk.size for ph in lv.phases for u in ph.units] for lv in self.levels]


def _gather_cols(A: sp.csc_matrix, cols: np.ndarray, active: np.ndarray):
    """Rows coupled to ``cols`` and the dense blocks ``A[cols,cols]``, ``A[rest,cols]``.

    Returns ``(rest, D_cc, D_rc)`` where ``rest`` are the active row indices
    outside ``cols`` carrying a nonzero in ``A[:, cols]`` (ascending).
    """
    if cols.size == 0:
        return np.zeros(0, np.int64), np.zeros((0, 0)), np.zeros((0, 0))
    ip, ix, dv = A.indptr, A.indices, A.data
    rows = [ix[ip[c]:ip[c + 1]] for c in cols]
    vals = [dv[ip[c]:ip[c + 1]] for c in cols]
    lens = np.array([r.size for r in rows])
    r_all = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    v_all = np.concatenate(vals) if vals else np.zeros(0)
    c_all = np.repeat(np.arange(cols.size), lens)
    keep = (v_all != 0.0) & active[r_all]
    r_all, v_all, c_all = r_all[keep], v_all[keep], c_all[keep]
    in_cols = np.isin(r_all, cols)
    rest = np.unique(r_all[~in_cols])
    pos_c = {int(g): i for i, g in enumerate(cols)}
    D_cc = np.zeros((cols.size, cols.size))
    D_rc = np.zeros((rest.size, cols.size))
    ri = r_all[in_cols]
    D_cc[np.array([pos_c[int(g)] for g in ri], dtype=np.int64), c_all[in_cols]] = v_all[in_cols]
    if rest.size:
        D_rc[np.searchsorted(rest, r_all[~in_cols]), c_all[~in_cols]] = v_all[~in_cols]
    return rest, D_cc, D_rc


def _mask(A: sp.csc_matrix, active: np.ndarray) -> sp.csc_matrix:
    D = sp.diags(active.astype(np.float64))
    out = (D @ A @ D).tocsc()
    out.eliminate_zeros()
    out.sort_indices()
    return out


def _coo(N, rows, cols, vals):
    if not rows:
        return sp.csc_matrix((N, N))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsc()


def _block(idx_r, idx_c, M):
    r = np.repeat(idx_r, idx_c.size)
    c = np.tile(idx_c, idx_r.size)
    return r, c, np.asarray(M).ravel()


def _precondition(A, active, grps, N, where, diagonal=False):
    """Block Jacobi preconditioning, Sec. 2.3: A <- C^T A C, C = diag(L_g^{-T}),
    L_g = chol(A_gg).  ``diagonal``: the local preconditioner of the concluding
    section that replaces block Cholesky by the diagonal, L_g = diag(A_gg)^{1/2}."""
    recs = []
    rows, cols, vals = [], [], []
    covered = np.zeros(N, dtype=bool)
    for key, t, g in grps:
        _, Agg, _ = _gather_cols(A, g, active)
        try:
            if diagonal:
                dg = np.diag(Agg)
                if not np.all(dg > 0.0):
                    raise NotSPD("nonpositive diagonal")
                Lg = np.diag(np.sqrt(dg))
            else:
                Lg = cholesky(Agg)
        except NotSPD:
            raise NotSPD(f"{where}: preconditioning block {key} not SPD") from None
        recs.append(GroupRec(g, Lg))
        Ci = ltsolve(Lg, np.eye(g.size))   # L_g^{-T}
        r, c, v = _block(g, g, Ci)
        rows.append(r); cols.append(c); vals.append(v)
        covered[g] = True
    rest = np.nonzero(~covered)[0]
    rows.append(rest); cols.append(rest); vals.append(np.ones(rest.size))
    C = _coo(N, rows, cols, vals)
    A = (C.T @ A @ C).tocsc()
    A.eliminate_zeros()
    A.sort_indices()
    return A, recs


def _skeletonize(A, active, units, tol, N, where, ties):
    """Skeletonization of every unit, Sec. 2.2, IDs first (parallel order)."""
    plans = []
    for key, t, e in units:
        Rr, Aee, ARe = _gather_cols(A, e, active)
        log = []
        k, perm, T = interp_decomp(ARe, tol, log)
        for (step, col, ncand) in log:
            ties.append((where, key, step, col, ncand))
        plans.append((key, e, Aee, k, perm, T))
    recs = []
    rows, cols, vals = [], [], []
    for key, e, Aee, k, perm, T in plans:
        s_loc, r_loc = perm[:k], perm[k:]
        sk, rd = e[s_loc], e[r_loc]
        A_rr = Aee[np.ix_(r_loc, r_loc)]
        A_sr = Aee[np.ix_(s_loc, r_loc)]
        A_ss = Aee[np.ix_(s_loc, s_loc)]
        # zeroing Z_I (Eq. 2.2): only the (rd, rd) and (sk, rd) blocks change
        At_rr = A_rr - T.T @ A_sr - A_sr.T @ T + T.T @ A_ss @ T
        At_sr = A_sr - A_ss @ T
        try:
            Lr = cholesky(At_rr)
        except NotSPD:
            raise NotSPD(f"{where}: skeleton block {key} not SPD") from None
        Xr = lsolve(Lr, At_sr.T)
        recs.append(SkelRec(e, sk, rd, T, Lr, Xr, key))
        if k and rd.size:
            r, c, v = _block(sk, sk, -(Xr.T @ Xr))
            rows.append(r); cols.append(c); vals.append(v)
        active[rd] = False
    A = (A + _coo(N, rows, cols, vals)).tocsc()
    return _mask(A, active), recs


def factor(A, ns, leaf: int, tol: float, precondition=True,
           edge_skel: bool = False, cell_order=None, snapshots: bool = False) -> Factor:
    """PHIF (``precondition=True``) or HIF (``False``) factorization of SPD ``A``.

    ``precondition="diag"``: PHIF with the diagonal local preconditioner of
    the concluding section in place of block Cholesky.

    ``cell_order``: optional callable ``(level, n_cells) -> permutation`` to
    process the cells of a level in another order (the result must not change,
    Sec. 2.1).  ``snapshots`` keeps ``A_l, A_l', A_l'', A_{l+1}`` per level
    (tiny grids only).
    """
    ns = tuple(int(n) for n in ns)
    d = len(ns)
    N = A.shape[0]
    diagonal = precondition == "diag"
    L = tree.num_levels(ns, leaf)
    A = sp.csc_matrix(A, dtype=np.float64, copy=True)
    A.sort_indices()
    active = np.ones(N, dtype=bool)
    levels, ties, snaps = [], [], []
    for lvl in range(L):
        width = leaf << lvl
        snap = {"A": A.copy()} if snapshots else None
        grps = tree.groups(ns, np.nonzero(active)[0], width)
        cells = [g for g in grps if g[1] == 0]
        if cell_order is not None:
            cells = [cells[i] for i in cell_order(lvl, len(cells))]
        # 1. cell elimination (Sec. 2.1)
        crecs = []
        rows, cols, vals = [], [], []
        for key, t, I in cells:
            B, AII, ABI = _gather_cols(A, I, active)
            try:
                Lc = cholesky(AII)
            except NotSPD:
                raise NotSPD(f"level {lvl}: cell {key} not SPD") from None
            X = lsolve(Lc, ABI.T)
            crecs.append(CellRec(I, B, Lc, X))
            if B.size:
                r, c, v = _block(B, B, -(X.T @ X))
                rows.append(r); cols.append(c); vals.append(v)
        for cr in crecs:
            active[cr.I] = False
        A = _mask((A + _coo(N, rows, cols, vals)).tocsc(), active)
        if snapshots:
            snap["A1"] = A.copy()
        # 2.-3. preconditioning and skeletonization of edges (2D) / faces (3D)
        phases = []
        seps = tree.groups(ns, np.nonzero(active)[0], width)
        if precondition:
            A, grecs = _precondition(A, active, seps, N, f"level {lvl}", diagonal)
        else:
            grecs = []
        if snapshots:
            snap["A2"] = A.copy()
        units = [g for g in seps if g[1] == 1]
        A, srecs = _skeletonize(A, active, units, tol, N, f"level {lvl}", ties)
        phases.append(Phase(grecs, srecs))
        # 4.-5. optional 3D edge skeletonization (Remark 3.1)
        if d == 3 and edge_skel:
            seps2 = [g for g in tree.groups(ns, np.nonzero(active)[0], width) if g[1] >= 2]
            if precondition:
                A, grecs2 = _precondition(A, active, seps2, N, f"level {lvl} edges", diagonal)
            else:
                grecs2 = []
            units2 = [g for g in seps2 if g[1] == 2]
            A, srecs2 = _skeletonize(A, active, units2, tol, N, f"level {lvl} edges", ties)
            phases.append(Phase(grecs2, srecs2))
        if snapshots:
            snap["A3"] = A.copy()
            snaps.append(snap)
        levels.append(Level(crecs, phases, int(active.sum())))
    S = np.nonzero(active)[0]
    _, ASS, _ = _gather_cols(A, S, active)
    try:
        BL = cholesky(ASS)
    except NotSPD:
        raise NotSPD("root block not SPD") from None
    return Factor(N, ns, leaf, tol, precondition, levels, S, BL, ties,
                  snaps if snapshots else None)


# ---------------------------------------------------------------------------
# application (Eqs. 3.1-3.3)
# ---------------------------------------------------------------------------

def solve(F: Factor, b: np.ndarray) -> np.ndarray:
    """``F^{-1} b = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T b`` (Eq. 3.2)."""
    x = np.array(b, dtype=np.float64, copy=True)
    for lv in F.levels:
        # E_l^T: per cell  y = L^{-1} x_I ; x_B -= X^T y ; x_I = y
        for c in lv.cells:
            y = lsolve(c.L, x[c.I])
            if c.B.size:
                x[c.B] -= c.X.T @ y
            x[c.I] = y
        for ph in lv.phases:
            for g in ph.groups:            # C^T: x_g = L_g^{-1} x_g
                x[g.g] = lsolve(g.L, x[g.g])
            for u in ph.units:             # K^T = E_rd^T Z^T
                if u.rd.size == 0:
                    continue
                xr = x[u.rd] - u.T.T @ x[u.sk]
                y = lsolve(u.L, xr)
                x[u.sk] -= u.X.T @ y
                x[u.rd] = y
    if F.S.size:
        x[F.S] = ltsolve(F.BL, lsolve(F.BL, x[F.S]))
    for lv in reversed(F.levels):
        for ph in reversed(lv.phases):
            for u in ph.units:             # K = Z E_rd
                if u.rd.size == 0:
                    continue
                xr = ltsolve(u.L, x[u.rd] - u.X @ x[u.sk])
                x[u.rd] = xr
                x[u.sk] -= u.T @ xr
            for g in ph.groups:            # C: x_g = L_g^{-T} x_g
                x[g.g] = ltsolve(g.L, x[g.g])
        for c in lv.cells:                 # E: x_I = L^{-T}(x_I - X x_B)
            r = x[c.I] - (c.X @ x[c.B] if c.B.size else 0.0)
            x[c.I] = ltsolve(c.L, r)
    return x


def matvec(F: Factor, b: np.ndarray) -> np.ndarray:
    """``F b = R_0^{-T} ... R_{L-1}^{-T} A_L R_{L-1}^{-1} ... R_0^{-1} b`` (Eq. 3.1)."""
    x = np.array(b, dtype=np.float64, copy=True)
    for lv in F.levels:                    # R_l^{-1} = K^{-1} C^{-1} E^{-1}
        for c in lv.cells:                 # E^{-1}: x_I = L^T x_I + X x_B
            x[c.I] = c.L.T @ x[c.I] + (c.X @ x[c.B] if c.B.size else 0.0)
        for ph in lv.phases:
            for g in ph.groups:            # C^{-1}: x_g = L_g^T x_g
                x[g.g] = g.L.T @ x[g.g]
            for u in ph.units:             # K^{-1} = E_rd^{-1} Z^{-1}
                if u.rd.size == 0:
                    continue
                x[u.sk] += u.T @ x[u.rd]
                x[u.rd] = u.L.T @ x[u.rd] + u.X @ x[u.sk]
    if F.S.size:
        x[F.S] = F.BL @ (F.BL.T @ x[F.S])
    for lv in reversed(F.levels):          # R_l^{-T} = E^{-T} C^{-T} K^{-T}
        for ph in reversed(lv.phases):
            for u in ph.units:             # K^{-T} = Z^{-T} E_rd^{-T}
                if u.rd.size == 0:
                    continue
                xr = x[u.rd].copy()
                x[u.sk] += u.X.T @ xr
                x[u.rd] = u.L @ xr
                x[u.rd] += u.T.T @ x[u.sk]
            for g in ph.groups:
                x[g.g] = g.L @ x[g.g]
        for c in lv.cells:                 # E^{-T}: x_B += X^T x_I ; x_I = L x_I
            xi = x[c.I].copy()
            if c.B.size:
                x[c.B] += c.X.T @ xi
            x[c.I] = c.L @ xi
    return x


# ---------------------------------------------------------------------------
# PCG and error estimators (Sec. 4)
# ---------------------------------------------------------------------------

def pcg(A, f: np.ndarray, M=None, rtol: float = 1e-12, maxit: int = 1000):
    """Preconditioned CG (Hestenes-Stiefel), x0 = 0, stopped on the recursive
    residual ``||r||/||f|| <= rtol``.  Returns ``(u, iters, true relres)``."""
    f = np.asarray(f, dtype=np.float64)
    x = np.zeros_like(f)
    r = f.copy()
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return x, 0, 0.0
    z = M(r) if M is not None else r.copy()
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = A @ p
        pq = float(p @ q)
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= rtol * nf:
            break
        z = M(r) if M is not None else r.copy()
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, float(np.linalg.norm(f - A @ x) / nf)


def power_norm(op, opT, n: int, seed: int = 0, rel: float = 1e-2, maxit: int = 100) -> float:
    """Randomized power iteration for ``||M||_2`` on ``M^T M`` (Sec. 4 estimator)."""
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal(n)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(maxit):
        w = opT(op(v))
        nw = np.linalg.norm(w)
        new = np.sqrt(nw)
        if nw == 0.0:
            return 0.0
        v = w / nw
        if est > 0 and abs(new - est) <= rel * new:
            return new
        est = new
    return est


def apply_error(A, F: Factor, seed: int = 0) -> float:
    """``e_a = ||A - F|| / ||A||`` (Sec. 4)."""
    n = A.shape[0]
    num = power_norm(lambda v: A @ v - matvec(F, v), lambda v: A @ v - matvec(F, v), n, seed)
    den = power_norm(lambda v: A @ v, lambda v: A @ v, n, seed + 1)
    return num / den


def solve_error(A, F: Factor, seed: int = 0) -> float:
    """``e_s = ||I - A F^{-1}||`` (Sec. 4)."""
    n = A.shape[0]
    return power_norm(lambda v: v - A @ solve(F, v), lambda v: v - solve(F, A @ v), n, seed)


def stats(F: Factor) -> dict:
    return {
        "levels": len(F.levels),
        "root": int(F.S.size),
        "active_after": [lv.active_after for lv in F.levels],
        "ranks": F.ranks,
        "ties": len(F.ties),
    }
