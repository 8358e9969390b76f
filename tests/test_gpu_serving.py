"""GPU tests of the serving patterns: differentiation (adjoint solve with the
stored factor), batched factor/PCG over many problems, plain HIF mode and a
larger 3D case, each against the FP64 oracle or a brute-force reference."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _loss_and_grad(lib, ns, log_a, f, u_obs, **opts):
    la = _dev(log_a).requires_grad_(True)
    ff = _dev(f).requires_grad_(True)
    u = lib.rhif_solve(la, ff, ns, **opts)
    loss = 0.5 * torch.sum((u - _dev(u_obs)) ** 2)
    loss.backward()
    return float(loss.detach()), la.grad.cpu().numpy(), ff.grad.cpu().numpy()


def test_autograd_gradient_matches_adjoint_formula_and_central_differences(gpu_lib):
    ns = (63, 63)
    log_star = W.gaussian_bump_log_field(ns, seed=5)
    log_a = 0.3 * W.gaussian_bump_log_field(ns, seed=6)
    f = np.ones(int(np.prod(ns)))
    A_star = fd.assemble(ns, np.exp(log_star), 0.0).tocsc()
    u_obs = spla.spsolve(A_star, f)
    opts = dict(leaf=16, tol=1e-6, precision="fp64", rtol=1e-13)
    loss, g, gf = _loss_and_grad(gpu_lib, ns, log_a, f, u_obs, **opts)
    # brute-force reference: sparse direct solves and the adjoint formula
    A = fd.assemble(ns, np.exp(log_a), 0.0).tocsc()
    u = spla.spsolve(A, f)
    lam = spla.spsolve(A, u - u_obs)
    g_ref = fd.dA_dlog_a(ns, np.exp(log_a), u, lam)
    assert abs(loss - 0.5 * np.sum((u - u_obs) ** 2)) <= 1e-9 * loss
    assert np.linalg.norm(g - g_ref) <= 1e-7 * np.linalg.norm(g_ref)
    assert np.linalg.norm(gf - lam) <= 1e-7 * np.linalg.norm(lam)
    # central differences of the loss computed by the GPU solver along random directions
    rng = np.random.default_rng(7)
    delta = 1e-4
    for _ in range(4):
        d = rng.standard_normal(log_a.shape)
        d /= np.linalg.norm(d)
        lp = _loss_and_grad(gpu_lib, ns, log_a + delta * d, f, u_obs, **opts)[0]
        lm = _loss_and_grad(gpu_lib, ns, log_a - delta * d, f, u_obs, **opts)[0]
        fdv = (lp - lm) / (2 * delta)
        assert abs(fdv - float(np.sum(g * d))) <= 1e-6 * max(abs(fdv), 1e-3 * loss)


def test_batched_factor_and_pcg_match_single_problem_runs(gpu_lib):
    sides = [31, 47, 64, 70, 39]
    nrhs = 4
    csrs, grids, fs, As = [], [], [], []
    for i, s in enumerate(sides):
        ns = (s, s)
        a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=100 + i)
        As.append(fd.assemble(ns, a, 0.0).tocsc())
        csrs.append(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0))
        grids.append(ns)
        fs.append(_dev(W.normal_rhs(ns, 200 + i, nrhs=nrhs)))
    facs, streams = gpu_lib.rhif_factor_batched(csrs, grids, 8, 1e-3, precision="fp32")
    us, its, rr = gpu_lib.rhif_pcg_batched(facs, fs, rtol=1e-10, streams=streams)
    torch.cuda.synchronize()
    for i, s in enumerate(sides):
        single = gpu_lib.rhif_factor(csrs[i], grids[i], 8, 1e-3, precision="fp32")
        lv = facs[i].stats()["levels"]
        assert [facs[i].skeletons(l) for l in range(lv)] == [single.skeletons(l) for l in range(lv)]
        x = fs[i][0].contiguous()
        np.testing.assert_array_equal(facs[i].apply(x).cpu().numpy(), single.apply(x).cpu().numpy())
        U = us[i].cpu().numpy()
        for r in range(nrhs):
            assert rr[i][r] <= 1.5e-10
            ud = spla.spsolve(As[i], fs[i][r].cpu().numpy())
            assert np.linalg.norm(U[r] - ud) <= 1e-7 * np.linalg.norm(ud)
        single.free()
        facs[i].free()


def test_hif_mode_matches_oracle(gpu_lib):
    ns = (63, 63)
    a = W.paper_quantized_field(ns, seed=4)
    A = fd.assemble(ns, a, 0.0)
    Fo = phif.factor(A, ns, 8, 1e-6, precondition=False)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, 8, 1e-6,
                             precision="fp64", precondition=False)
    for lvl in range(len(Fo.levels)):
        go = {frozenset(map(int, u.e)): frozenset(map(int, u.sk)) for u in Fo.levels[lvl].phases[0].units}
        gg = {frozenset(map(int, d)): frozenset(map(int, d[:k])) for d, k in Fg.skeletons(lvl)}
        assert go == gg or Fo.ties
    x = np.random.default_rng(3).standard_normal(A.shape[0])
    yo = phif.solve(Fo, x)
    yg = Fg.apply(_dev(x)).cpu().numpy()
    if not Fo.ties:
        assert np.linalg.norm(yg - yo) <= 1e-8 * np.linalg.norm(yo)


@pytest.mark.parametrize("edge", [False, True])
def test_3d_31cube_matches_oracle(gpu_lib, edge):
    ns, leaf = (31, 31, 31), 8
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=sum(ns) + leaf)
    A = fd.assemble(ns, a, 1e-2)
    Fo = phif.factor(A, ns, leaf, 1e-3, edge_skel=edge)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 1e-2), ns, leaf, 1e-3,
                             precision="fp64", edge_skel_3d=edge)
    same = True
    for lvl in range(len(Fo.levels)):
        for p in range(len(Fo.levels[lvl].phases)):
            go = {frozenset(map(int, u.e)): frozenset(map(int, u.sk)) for u in Fo.levels[lvl].phases[p].units}
            gg = {frozenset(map(int, d)): frozenset(map(int, d[:k])) for d, k in Fg.skeletons(lvl, p)}
            assert set(go) == set(gg)
            same &= go == gg
    assert same or Fo.ties
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    yo = phif.solve(Fo, x)
    yg = Fg.apply(_dev(x)).cpu().numpy()
    if same:
        assert np.linalg.norm(yg - yo) <= 1e-9 * np.linalg.norm(yo)
    f = W.normal_rhs(ns, 9)
    u, its, rr = Fg.pcg(_dev(f), rtol=1e-10)
    assert rr[0] <= 1.5e-10
    # the FP32 factor converges to the same solution
    F32 = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 1e-2), ns, leaf, 1e-3,
                              precision="fp32", edge_skel_3d=edge)
    u32, its32, rr32 = F32.pcg(_dev(f), rtol=1e-10)
    assert rr32[0] <= 1.5e-10
    assert float(torch.linalg.norm(u32 - u) / torch.linalg.norm(u)) <= 1e-8
