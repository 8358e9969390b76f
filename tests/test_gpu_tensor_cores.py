"""The tensor-core tile product (tcgen05, FP32 accumulation) against an FP64
reference, for each operand kind, and the mixed-precision factors that use it
for the Schur updates of large fronts (Sec. 2.1) against the FP64 oracle.

Bars of the tile product, elementwise with S = sum_k |a_ik| |b_jk|:
 * TF32 split (three products): |C_tc - C_ref| <= 2e-6 S + 1e-6 |C_ref|: the
   split keeps about 2^-21 relative error per product and FP32 accumulation
   adds ~K 2^-24, so plain TF32 inputs (error ~2^-11 per product) fail it;
 * TF32: <= 2^-10 S (each operand rounded to nearest TF32, 2^-11 relative)
   + 1e-6 |C_ref|;
 * BF16: <= 2^-8 S (each operand rounded to nearest BF16, 2^-9 relative)
   + 1e-6 |C_ref|.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fd, phif

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BARS = {"tf32x3": 2e-6, "tf32": 2.0 ** -10, "bf16": 2.0 ** -8}


def _colmajor(a):
    return torch.as_tensor(np.asfortranarray(a), device="cuda")


def _case(M, N, K):
    g = np.random.default_rng(M * 1000 + N + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    C = g.standard_normal((M, N)).astype(np.float32)
    ref = C.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    return A, B, C, ref, bound


@pytest.mark.parametrize("kind", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (256, 128, 96), (100, 50, 37), (384, 192, 1000),
                                   (130, 70, 0), (1, 1, 5), (128, 64, 16)])
def test_tc_gemm_matches_fp64(gpu_lib, kind, M, N, K):
    A, B, C, ref, bound = _case(M, N, K)
    Cd = _colmajor(C)
    assert Cd.stride(0) == 1
    gpu_lib.rhif_tc_gemm_check(_colmajor(A), _colmajor(B), Cd, kind=kind)
    out = Cd.cpu().numpy().astype(np.float64)
    err = np.abs(out - ref)
    assert np.all(err <= BARS[kind] * bound + 1e-6 * np.abs(ref) + 1e-30)
    if kind != "tf32x3" and K >= 32:
        # the reduced kinds really round their inputs: they miss the split's bar
        assert np.any(err > BARS["tf32x3"] * bound + 1e-6 * np.abs(ref))


def test_tc_gemm_rejects_unknown_kind(gpu_lib):
    import ctypes
    C = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    rc = gpu_lib._lib.rhif_tc_gemm_check(7, 4, 4, 0, None, 4, None, 4,
                                         ctypes.c_void_p(C.data_ptr()), 4, None)
    assert rc == -1


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_mixed_factor_with_tensor_core_schur_against_fp64_oracle(gpu_lib, precision):
    """31^3, leaf 8, faces + edges: the level-1 fronts (about a thousand DOFs)
    take the many-CTA schedule whose Schur tiles run on the tensor cores with
    the chosen operands.  States ||F^{-1} x - Fo^{-1} x|| / ||Fo^{-1} x|| and
    the apply errors; PCG with the factor reaches relres 1e-10 and the direct
    solution."""
    ns = (31, 31, 31)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=W.SEED_BASE + 31)
    A = fd.assemble(ns, a, 1e-2)
    Fo = phif.factor(A, ns, 8, 1e-3, edge_skel=True)
    gpu_lib.rhif_reset_kernel_stats()
    Fg = gpu_lib.rhif_factor(gpu_lib.rhif_assemble_fd(ns, torch.as_tensor(a, device="cuda"), 1e-2),
                             ns, 8, 1e-3, precision=precision, edge_skel_3d=True)
    x = np.random.default_rng(3).standard_normal(A.shape[0])
    yo = phif.solve(Fo, x)
    yg = Fg.apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    diff = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    Ax = A @ x
    eg = np.linalg.norm(Fg.apply(torch.as_tensor(Ax, device="cuda")).cpu().numpy() - x) / np.linalg.norm(x)
    eo = np.linalg.norm(phif.solve(Fo, Ax) - x) / np.linalg.norm(x)
    f = W.normal_rhs(ns, 5)
    u, its, rr = Fg.pcg(torch.as_tensor(f, device="cuda"), rtol=1e-10, maxit=300)
    ud = spla.spsolve(A.tocsc(), f)
    du = np.linalg.norm(u.cpu().numpy() - ud) / np.linalg.norm(ud)
    print(f"\n31^3 {precision} factor: |F^-1x - Fo^-1x|/|Fo^-1x| = {diff:.3e}, apply err {eg:.3e} "
          f"(oracle {eo:.3e}), pcg its {its[0]}, |u - u_direct|/|u_direct| = {du:.2e}")
    assert rr[0] <= 1.5e-10 and du <= 1e-7
    assert eg <= 2 * eo + {"fp32": 1e-3, "tf32": 0.5, "bf16": 1.0}[precision]
    Fg.free()
