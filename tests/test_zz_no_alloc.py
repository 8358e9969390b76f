"""rhif_apply_noalloc: F^{-1} x with no device allocation, for callers that
cannot allocate while they apply the preconditioner (an outer solver that has
reserved all device memory, or code that must not risk the synchronization or
the mid-run failure of an allocation).  Its output must equal rhif_apply's on
consecutive calls, and oversized requests must be refused before any work.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(lib, F, x, out):
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib._lib.rhif_apply_noalloc(F._h, nrhs, ctypes.c_void_p(x.data_ptr()), F.N,
                                       ctypes.c_void_p(out.data_ptr()), F.N, s)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_apply_matches_apply_on_consecutive_calls(gpu_lib, precision):
    ns = (255, 255)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=21)
    csr = gpu_lib.rhif_assemble_fd(ns, torch.as_tensor(a, device="cuda"), 0.0)
    F = gpu_lib.rhif_factor(csr, ns, 8, 1e-3, precision=precision)
    for call in range(2):
        x = torch.as_tensor(W.normal_rhs(ns, 40 + call, nrhs=2), device="cuda")
        ref = F.apply(x)
        out = torch.full_like(x, float("nan"))
        assert _noalloc(gpu_lib, F, x, out) == 0
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r)
    F.free()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_apply_matches_apply_with_many_cta_fronts(gpu_lib, precision):
    """3D factor with every front eliminated by the many-CTA schedule
    (big_front = 1): its sweeps use the interior part of the scratch too."""
    ns = (15, 15, 15)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=23)
    csr = gpu_lib.rhif_assemble_fd(ns, torch.as_tensor(a, device="cuda"), 1e-2)
    F = gpu_lib.rhif_factor(csr, ns, 4, 1e-3, precision=precision, edge_skel_3d=True, big_front=1)
    for call in range(2):
        x = torch.as_tensor(W.normal_rhs(ns, 50 + call, nrhs=3), device="cuda")
        ref = F.apply(x)
        out = torch.full_like(x, float("nan"))
        assert _noalloc(gpu_lib, F, x, out) == 0
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r)
    F.free()


def test_noalloc_rejects_requests_beyond_the_static_scratch(gpu_lib):
    ns = (255, 255)
    a = W.log_uniform_pixels(ns, 1e-3, 1e3, seed=22)
    csr = gpu_lib.rhif_assemble_fd(ns, torch.as_tensor(a, device="cuda"), 0.0)
    F = gpu_lib.rhif_factor(csr, ns, 8, 1e-3, precision="fp32")
    nrhs = 64   # about 2x the boundary contributions the 2^20-entry scratch holds
    x = torch.zeros((nrhs, F.N), dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    assert _noalloc(gpu_lib, F, x, out) == -1
    assert b"static scratch" in gpu_lib._lib.rhif_last_error_detail()
    F.free()
