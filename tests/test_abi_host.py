"""Host-side behaviour of the C ABI (include/rhif.h) on the CPU: the argument
checks every entry point makes before it touches the GPU, the error strings,
the default options and the stored-entry count of the finite-difference
matrix (against the oracle's assembly, Eqs. 1.1-1.2).  No device call is
made: every call here returns before its first CUDA runtime call."""
import ctypes
import math

import numpy as np
import pytest

import workloads as W
from oracle import fd

pytestmark = pytest.mark.filterwarnings("ignore")

OK, BAD_ARG = 0, -1


@pytest.fixture(scope="module")
def rhif():
    import os
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build the library")
    import paper_1808_01364_gb300 as r
    r.load()
    return r


def _grid(rhif, ns):
    return ctypes.byref(rhif._grid(ns))


def _csr(rhif, nrows, nnz):
    # host addresses standing in for device pointers: the checks below never
    # dereference them
    buf = (ctypes.c_double * 4)()
    p = ctypes.addressof(buf)
    return rhif.CSR(nrows, nnz, p, p, p), buf


@pytest.mark.parametrize("ns", [(1, 1), (1, 7), (5, 3), (31, 17), (2, 2, 2), (9, 8, 7), (1, 1, 6)])
def test_fd_nnz_counts_the_oracles_stored_entries(rhif, ns):
    A = fd.assemble(ns, np.ones(W.pixel_shape(ns)), 0.0)
    assert rhif._lib.rhif_fd_nnz(_grid(rhif, ns)) == A.nnz


def test_fd_nnz_rejects_bad_grids(rhif):
    g = rhif.Grid(4, (ctypes.c_int * 3)(3, 3, 3))
    assert rhif._lib.rhif_fd_nnz(ctypes.byref(g)) == -1
    assert rhif._lib.rhif_fd_nnz(_grid(rhif, (0, 5))) == -1
    assert rhif._lib.rhif_fd_nnz(None) == -1


def test_default_options(rhif):
    o = rhif.Opts()
    ctypes.memset(ctypes.byref(o), 0x5A, ctypes.sizeof(o))
    assert rhif._lib.rhif_default_opts(ctypes.byref(o)) == OK
    assert (o.precision, o.precondition, o.edge_skel_3d) == (rhif.RHIF_FP64, 1, 0)
    assert (o.big_front, o.big_frame, o.skel_cluster, o.tensor_cores) == (0, 0, 0, 0)
    assert rhif._lib.rhif_default_opts(None) == BAD_ARG


def test_error_strings(rhif):
    for code, name in rhif.ERRORS.items():
        want = "RHIF_OK" if code == 0 else f"RHIF_ERR_{name}"
        assert rhif._lib.rhif_error_string(code).decode() == want
    assert rhif._lib.rhif_error_string(-12345)


def test_factor_rejects_bad_arguments_before_any_device_work(rhif):
    lib = rhif._lib
    ns = (15, 15)
    N = 15 * 15
    h = ctypes.c_void_p(1234)
    A, _keep = _csr(rhif, N, 5 * N)
    o = rhif._opts()

    def call(A_=ctypes.byref(A), g=_grid(rhif, ns), leaf=4, tol=1e-3, opts=ctypes.byref(o),
             out=ctypes.byref(h)):
        return lib.rhif_factor(A_, g, leaf, tol, opts, None, out)

    assert call(out=None) == BAD_ARG
    assert call(g=_grid(rhif, (0, 15))) == BAD_ARG
    assert call(A_=None) == BAD_ARG
    assert call(leaf=1) == BAD_ARG
    assert call(tol=-1e-3) == BAD_ARG
    assert call(tol=math.nan) == BAD_ARG
    assert call(tol=math.inf) == BAD_ARG
    bad = rhif._opts()
    bad.precision = 7
    assert call(opts=ctypes.byref(bad)) == BAD_ARG
    for v in (-1, 3):   # 0 HIF, 1 block Jacobi, 2 diagonal
        bad = rhif._opts()
        bad.precondition = v
        assert call(opts=ctypes.byref(bad)) == BAD_ARG
    wrong_rows, _k2 = _csr(rhif, N - 1, 5 * N)
    assert call(A_=ctypes.byref(wrong_rows)) == BAD_ARG
    too_few, _k3 = _csr(rhif, N, N - 1)
    assert call(A_=ctypes.byref(too_few)) == BAD_ARG
    for sc in (3, 32, 6):
        c = rhif._opts(skel_cluster=sc)
        assert call(opts=ctypes.byref(c)) == BAD_ARG
    assert h.value is None      # the output handle is cleared on failure
    assert lib.rhif_last_error_detail().decode()


def test_handle_calls_reject_a_null_handle(rhif):
    lib = rhif._lib
    buf = (ctypes.c_double * 8)()
    p = ctypes.addressof(buf)
    it = (ctypes.c_int * 1)()
    rr = (ctypes.c_double * 1)()
    es = ctypes.c_double()
    n = ctypes.c_int()
    assert lib.rhif_apply(None, rhif.RHIF_SOLVE, 1, p, 8, p, 8, None) == BAD_ARG
    assert lib.rhif_apply_noalloc(None, 1, p, 8, p, 8, None) == BAD_ARG
    assert lib.rhif_spmv(None, 1, p, 8, p, 8, None) == BAD_ARG
    assert lib.rhif_pcg(None, 1, p, 8, p, 8, 1e-10, 10, it, rr, None) == BAD_ARG
    assert lib.rhif_estimate_es(None, p, 10, 1e-2, ctypes.byref(es), ctypes.byref(n), None) == BAD_ARG
    assert lib.rhif_stats(None, ctypes.byref(rhif.Stats())) == BAD_ARG
    assert lib.rhif_skeletons(None, 0, 0, ctypes.byref(n), None, None, None, 0) == BAD_ARG
    lib.rhif_free(None)          # a no-op


def test_other_entry_points_check_their_arguments(rhif):
    lib = rhif._lib
    buf = (ctypes.c_double * 8)()
    p = ctypes.addressof(buf)
    A, _keep = _csr(rhif, 225, 1125)
    # rhif_autotune needs somewhere to put its answer
    assert lib.rhif_autotune(ctypes.byref(A), _grid(rhif, (15, 15)), 4, 1e-3, None, 10, None,
                             None, None) == BAD_ARG
    best = rhif.Opts()
    assert lib.rhif_autotune(ctypes.byref(A), _grid(rhif, (15, 15)), 4, 1e-3, None, -1, None,
                             ctypes.byref(best), None) == BAD_ARG
    # assembly and gradient: bad grids and null pointers
    assert lib.rhif_assemble_fd(_grid(rhif, (0, 3)), p, None, 0.0, p, p, p, None) == BAD_ARG
    assert lib.rhif_assemble_fd(_grid(rhif, (3, 3)), None, None, 0.0, p, p, p, None) == BAD_ARG
    assert lib.rhif_grad_logcoef(_grid(rhif, (3, 3)), p, p, None, p, None) == BAD_ARG
    # tensor-core check: operand kind and shapes
    assert lib.rhif_tc_gemm_check(0, 0, 4, 4, p, 4, p, 4, p, 4, None) == BAD_ARG
    assert lib.rhif_tc_gemm_check(2, 4, 4, 4, p, 3, p, 4, p, 4, None) == BAD_ARG
    assert lib.rhif_tc_gemm_check(3, 4, 4, 4, p, 4, p, 4, p, 4, None) == BAD_ARG
    assert lib.rhif_tc_gemm_check(-1, 4, 4, 4, p, 4, p, 4, p, 4, None) == BAD_ARG
    # batches: negative counts and missing streams
    out = (ctypes.c_void_p * 1)()
    assert lib.rhif_factor_batched(-1, ctypes.byref(A), _grid(rhif, (15, 15)), 4, 1e-3, None,
                                   None, 1, out) == BAD_ARG
    assert lib.rhif_pcg_batched(1, None, 1, None, None, 1e-10, 10, None, None, None, 1) == BAD_ARG
    # kernel statistics: index range
    st = rhif.KernelStat()
    assert lib.rhif_kernel_stats(-1, ctypes.byref(st)) == BAD_ARG
    assert lib.rhif_kernel_stats(lib.rhif_kernel_stat_count(), ctypes.byref(st)) == BAD_ARG


def test_binding_checks_buffer_sizes_before_the_device(rhif):
    """The C ABI takes bare pointers, so the binding refuses tensors whose
    sizes do not match the grid (a short buffer would be read or written
    out of bounds on the GPU)."""
    import torch
    ns = (15, 15)
    N, npix = 15 * 15, 16 * 16
    with pytest.raises(ValueError, match="a_pix"):
        rhif.rhif_assemble_fd(ns, torch.ones(npix - 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="b"):
        rhif.rhif_assemble_fd(ns, torch.ones(npix, dtype=torch.float64), torch.ones(N + 1))
    with pytest.raises(ValueError, match="log_a_pix"):
        rhif.rhif_assemble_fd_log(ns, torch.zeros(npix + 3, dtype=torch.float64))
    nnz = 5 * N - 4 * 15
    good = (torch.zeros(N + 1, dtype=torch.int64), torch.zeros(nnz, dtype=torch.int32),
            torch.zeros(nnz, dtype=torch.float64))
    for bad, what in [((good[0][:-1], good[1], good[2]), "rowptr"),
                      ((good[0], good[1][:-1], good[2]), "col"),
                      ((good[0], good[1].long(), good[2]), "col"),
                      ((good[0], good[1], good[2].float()), "val")]:
        with pytest.raises(ValueError, match=what):
            rhif.rhif_factor(bad, ns, 4, 1e-3)
        with pytest.raises(ValueError, match=what):
            rhif.rhif_autotune(bad, ns, 4, 1e-3)
    with pytest.raises(ValueError, match="CUDA"):
        rhif.rhif_factor(good, ns, 4, 1e-3)       # right sizes, but host memory
    u = torch.zeros(N, dtype=torch.float64)
    with pytest.raises(ValueError, match="lam"):
        rhif.rhif_grad_logcoef(ns, torch.ones(npix, dtype=torch.float64), u, u[:-1])
    with pytest.raises(ValueError, match="a_pix"):
        rhif.rhif_grad_logcoef(ns, torch.ones(npix, dtype=torch.float32), u, u)
