"""GPU error estimator e_s = ||I - A F^{-1}||_2 (Sec. 4) against the oracle,
and the paper's PHIF-vs-HIF comparison on its high-contrast field.

Parity: both sides run the same power iteration (the oracle's power_norm)
from the same seeded start vector for a fixed number of M^T M products
(rel = 0), with the FP64 factor whose skeletons match the oracle's, so the
estimates agree to rounding (1e-8 relative).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _start(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal(n)


@pytest.mark.parametrize("ns,leaf,tol,precondition", [
    ((63, 63), 8, 1e-3, True),
    ((63, 63), 8, 1e-3, False),
    ((15, 15, 15), 4, 1e-3, True),
])
def test_es_matches_oracle_power_iteration(gpu_lib, ns, leaf, tol, precondition):
    a = W.paper_quantized_field(ns, seed=3)
    A = fd.assemble(ns, a, 0.0)
    Fo = phif.factor(A, ns, leaf, tol, precondition=precondition)
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0), ns, leaf, tol,
                             precision="fp64", precondition=precondition)
    n = A.shape[0]
    seed, iters = 11, 12
    es_o = phif.power_norm(lambda v: v - A @ phif.solve(Fo, v),
                           lambda v: v - phif.solve(Fo, A @ v), n, seed, rel=0.0, maxit=iters)
    es_g, it_g = Fg.estimate_es(_dev(_start(n, seed)), maxit=iters, rel=0.0)
    assert it_g == iters
    if not Fo.ties:
        assert abs(es_g - es_o) <= 1e-8 * es_o
    # the default stopping rule (1e-2 relative change) lands within 2e-2
    es_s, _ = Fg.estimate_es(_dev(_start(n, seed)))
    assert abs(es_s - es_o) <= 2e-2 * es_o
    Fg.free()


def test_phif_beats_hif_on_the_paper_field(gpu_lib):
    """Sec. 4 (Tables 1-2): on the quantized high-contrast field, block Jacobi
    preconditioning makes the factor a much better preconditioner than plain
    HIF at the same tolerance (smaller e_s, fewer PCG iterations), or HIF
    breaks down (not SPD) where PHIF does not."""
    ns, leaf, tol = (255, 255), 16, 1e-3
    a = W.paper_quantized_field(ns, seed=21)
    csr = gpu_lib.rhif_assemble_fd(ns, _dev(a), 0.0)
    f = _dev(W.normal_rhs(ns, 22))
    x0 = _dev(_start(ns[0] * ns[1], 23))
    Fp = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp64", precondition=True)
    es_p, _ = Fp.estimate_es(x0)
    _, its_p, rr_p = Fp.pcg(f, rtol=1e-10)
    assert rr_p[0] <= 1.5e-10
    try:
        Fh = gpu_lib.rhif_factor(csr, ns, leaf, tol, precision="fp64", precondition=False)
    except gpu_lib.RhifError as e:
        assert e.code == -2
        return
    es_h, _ = Fh.estimate_es(x0)
    _, its_h, _ = Fh.pcg(f, rtol=1e-10, maxit=500, check=False)
    assert es_p < es_h
    assert its_p[0] <= its_h[0]
