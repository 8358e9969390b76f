"""The differentiation workload at full size: 511^2 coefficient recovery.

Loss 0.5 ||u(log a) - u_obs||^2, u_obs = A(log a*)^{-1} f with log a* a sum of
20 seeded Gaussian bumps of amplitude 3 and f = 1; the iterate is log a = 0
(constant a, the starting point of a recovery).  The gradient with respect to
the per-pixel log a comes from the autograd function: forward PCG, adjoint
PCG with the same stored factor (A is symmetric, Sec. 1), and the gradient
kernel.  It is checked

* against the FP64 oracle: the oracle's own factor (Sec. 3) as the
  preconditioner of the oracle's PCG for the state and the adjoint, and the
  oracle's per-pixel formula -lam^T (dA/dlog a_p) u;
* by central differences of the GPU loss along 64 seeded random directions;
* for the FP32 factor, against the same FP64 oracle gradient (stated).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NS = (511, 511)
OPTS = dict(leaf=16, tol=1e-6, rtol=1e-12)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def problem():
    log_star, f = W.inverse_problem(NS)
    A_star = fd.assemble(NS, np.exp(log_star), 0.0)
    Fo_star = phif.factor(A_star, NS, 16, 1e-6)
    u_obs, _, rr = phif.pcg(A_star, f, M=lambda r: phif.solve(Fo_star, r), rtol=1e-13)
    log_a = np.zeros_like(log_star)
    # oracle gradient at log a (FP64 factor as preconditioner, PCG to 1e-13)
    A = fd.assemble(NS, np.exp(log_a), 0.0)
    Fo = phif.factor(A, NS, 16, 1e-6)
    u, _, _ = phif.pcg(A, f, M=lambda r: phif.solve(Fo, r), rtol=1e-13)
    lam, _, _ = phif.pcg(A, u - u_obs, M=lambda r: phif.solve(Fo, r), rtol=1e-13)
    g_or = fd.dA_dlog_a(NS, np.exp(log_a), u, lam)
    loss_or = 0.5 * float(np.sum((u - u_obs) ** 2))
    return log_a, f, u_obs, g_or, loss_or


def _loss_grad(lib, log_a, f, u_obs, precision, grad=True):
    la = _dev(log_a).requires_grad_(grad)
    u = lib.rhif_solve(la, _dev(f), NS, precision=precision, **OPTS)
    loss = 0.5 * torch.sum((u - _dev(u_obs)) ** 2)
    if not grad:
        return float(loss.detach()), None
    loss.backward()
    return float(loss.detach()), la.grad.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gradient_matches_fp64_oracle(gpu_lib, problem, precision):
    log_a, f, u_obs, g_or, loss_or = problem
    loss, g = _loss_grad(gpu_lib, log_a, f, u_obs, precision)
    err = np.linalg.norm(g - g_or) / np.linalg.norm(g_or)
    print(f"\n511^2 gradient, {precision} factor: |g - g_oracle|/|g_oracle| = {err:.3e}, "
          f"loss {loss:.6e} (oracle {loss_or:.6e})")
    # both sides solve to relres 1e-12/1e-13; the solution error is the
    # amplification (~1e2 on this smooth field) times that, and the gradient
    # is bilinear in (u, lam)
    assert err <= 1e-8
    assert abs(loss - loss_or) <= 1e-8 * loss_or


def test_gradient_by_central_differences_on_64_directions(gpu_lib, problem):
    log_a, f, u_obs, _, _ = problem
    loss, g = _loss_grad(gpu_lib, log_a, f, u_obs, "fp64")
    rng = np.random.default_rng(W.SEED_BASE + 45)
    delta = 1e-4
    worst = worst_g = 0.0
    gn = np.linalg.norm(g)
    for _ in range(64):
        d = rng.standard_normal(log_a.shape)
        d /= np.linalg.norm(d)
        lp, _ = _loss_grad(gpu_lib, log_a + delta * d, f, u_obs, "fp64", grad=False)
        lm, _ = _loss_grad(gpu_lib, log_a - delta * d, f, u_obs, "fp64", grad=False)
        fdv = (lp - lm) / (2 * delta)
        gd = float(np.sum(g * d))
        worst = max(worst, abs(fdv - gd) / abs(fdv))
        worst_g = max(worst_g, abs(fdv - gd) / gn)
    print(f"\n511^2 central differences (delta {delta:g}, 64 directions): "
          f"max |fd - g.d| / |fd| = {worst:.3e}, max |fd - g.d| / |g| = {worst_g:.3e}; "
          f"|g| = {gn:.3e}, loss {loss:.6e}")
    assert worst_g <= 1e-6
