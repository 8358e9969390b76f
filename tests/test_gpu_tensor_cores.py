"""The tensor-core tile product (tcgen05, TF32 inputs split into a high part
and a remainder, FP32 accumulation) against an FP64 reference.

Bar: |C_tc - C_ref| <= 2e-6 * sum_k |a_ik| |b_jk| + 1e-6 |C_ref| elementwise;
the split keeps about 2^-21 relative error per product and FP32 accumulation
adds ~K * 2^-24, so plain TF32 inputs (error ~2^-11 per product) fail it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _colmajor(a):
    return torch.as_tensor(np.asfortranarray(a), device="cuda")


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (256, 128, 96), (100, 50, 37), (384, 192, 1000),
                                   (130, 70, 0), (1, 1, 5)])
def test_tc_gemm_matches_fp64(gpu_lib, M, N, K):
    g = np.random.default_rng(M * 1000 + N + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    C = g.standard_normal((M, N)).astype(np.float32)
    ref = C.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    Cd = _colmajor(C)
    assert Cd.stride(0) == 1
    gpu_lib.rhif_tc_gemm_check(_colmajor(A), _colmajor(B), Cd)
    out = Cd.cpu().numpy().astype(np.float64)
    err = np.abs(out - ref)
    assert np.all(err <= 2e-6 * bound + 1e-6 * np.abs(ref) + 1e-30)
