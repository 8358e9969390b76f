"""Python binding of librhif (include/rhif.h): argument marshalling only.

Every step of the factorization, the application of F^{-1} and PCG runs in the
CUDA library; this module passes torch device pointers and the current stream
through ctypes.  There is no CPU fallback: :func:`load` raises if the library
cannot be built or loaded, and every call raises :class:`RhifError` on a
non-zero return code.

Names follow the C ABI: ``rhif_assemble_fd``, ``rhif_factor`` (returns a
:class:`Factor` with ``apply``/``pcg``/``spmv``/``stats``/``skeletons``/``free``),
``rhif_grad_logcoef``, plus :class:`RhifSolve`, the torch.autograd function of
the differentiation workload.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lib = None
_lock = threading.Lock()

RHIF_FP64, RHIF_MIXED_FP32 = 0, 1
RHIF_SOLVE, RHIF_MATVEC, RHIF_HALF, RHIF_HALF_T = 0, 1, 2, 3
ERRORS = {0: "OK", -1: "BAD_ARG", -2: "NOT_SPD", -3: "NOT_CONVERGED", -4: "TIMEOUT", -5: "OOM",
          -6: "CUDA"}


class RhifError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__(f"RHIF_ERR_{ERRORS.get(code, code)}: {detail}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class CSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precondition", ctypes.c_int),
                ("edge_skel_3d", ctypes.c_int), ("big_front", ctypes.c_int),
                ("big_frame", ctypes.c_int), ("skel_cluster", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("leaf_fp64", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n", ctypes.c_int64), ("root_size", ctypes.c_int64),
                ("active", ctypes.c_int64 * 16), ("factor_bytes", ctypes.c_int64),
                ("flops", ctypes.c_double), ("apply_bytes", ctypes.c_double),
                ("precision", ctypes.c_int), ("units", ctypes.c_int),
                ("factor_ms", ctypes.c_double), ("fp64_leaves", ctypes.c_int),
                ("unit_dofs", ctypes.c_int64 * 16), ("skeletons", ctypes.c_int64 * 16)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


EXPORTS = {
    "rhif_default_opts": (ctypes.c_int, [ctypes.POINTER(Opts)]),
    "rhif_fd_nnz": (ctypes.c_int64, [ctypes.POINTER(Grid)]),
    "rhif_assemble_fd": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "rhif_assemble_fd_log": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rhif_factor": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.POINTER(Grid), ctypes.c_int,
                                   ctypes.c_double, ctypes.POINTER(Opts), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "rhif_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rhif_spmv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rhif_apply_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p]),
    "rhif_pcg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                ctypes.c_void_p]),
    "rhif_tc_gemm_check": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p]),
    "rhif_estimate_ea": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "rhif_estimate_es": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "rhif_grad_logcoef": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "rhif_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "rhif_skeletons": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "rhif_factor_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_double, ctypes.POINTER(Opts), ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "rhif_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "rhif_pcg_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "rhif_factor_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_double, ctypes.POINTER(Opts),
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rhif_pcg_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                        ctypes.c_int]),
    "rhif_autotune": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.POINTER(Grid), ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(Opts), ctypes.c_int,
                                     ctypes.c_void_p, ctypes.POINTER(Opts),
                                     ctypes.POINTER(ctypes.c_double)]),
    "rhif_plan_selfcheck": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                           ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "rhif_free": (None, [ctypes.c_void_p]),
    "rhif_set_timing": (ctypes.c_int, [ctypes.c_int]),
    "rhif_reset_kernel_stats": (ctypes.c_int, []),
    "rhif_kernel_stat_count": (ctypes.c_int, []),
    "rhif_kernel_stats": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(KernelStat)]),
    "rhif_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rhif_last_error_detail": (ctypes.c_char_p, []),
}


def load(rebuild: bool = False):
    """Load librhif.so, building it first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None and not rebuild:
            return _lib
        if rebuild or not _build.up_to_date():
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        raise RhifError(rc, _lib.rhif_last_error_detail().decode())


def _grid(ns) -> Grid:
    ns = [int(v) for v in ns]
    g = Grid()
    g.dim = len(ns)
    for i in range(3):
        g.n[i] = ns[i] if i < len(ns) else 1
    return g


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _colptr(t: torch.Tensor):
    """Pointer of a 2-D CUDA tensor stored column-major (unit row stride)."""
    assert t.is_cuda and t.dim() == 2 and (t.stride(0) == 1 or t.shape[0] <= 1 or
                                            t.numel() == 0), \
        "expected a column-major 2-D CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _cols(x: torch.Tensor, N: int):
    """(N,) or (nrhs, N) contiguous float64 -> (nrhs, ld)."""
    assert x.dtype == torch.float64 and x.is_cuda and x.is_contiguous()
    if x.dim() == 1:
        assert x.numel() == N
        return 1, N
    assert x.dim() == 2 and x.shape[1] == N
    return x.shape[0], N


def _npix(ns) -> int:
    n = 1
    for v in ns:
        n *= int(v) + 1
    return n


def _ndof(ns) -> int:
    n = 1
    for v in ns:
        n *= int(v)
    return n


def _need(t, name: str, numel: int, dtype=None):
    """Sizes are checked here because the C ABI takes bare device pointers:
    a short buffer would be read or written out of bounds on the GPU."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.numel() != numel:
        raise ValueError(f"{name}: {t.numel()} entries, expected {numel}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")


def _on_device(**tensors):
    for name, t in tensors.items():
        if not t.is_cuda:
            raise ValueError(f"{name}: expected a CUDA tensor")


def _csr(csr, ns) -> CSR:
    """CSR struct of (rowptr int64 [N+1], col int32 [nnz], val float64 [nnz]) on grid ns."""
    rowptr, col, val = csr
    N = _ndof(ns)
    _need(rowptr, "rowptr", N + 1, torch.int64)
    _need(col, "col", val.numel(), torch.int32)
    _need(val, "val", col.numel(), torch.float64)
    _on_device(rowptr=rowptr, col=col, val=val)
    for t in csr:
        assert t.is_contiguous(), "CSR arrays must be contiguous"
    return CSR(N, val.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())


def rhif_fd_nnz(ns) -> int:
    load()
    return int(_lib.rhif_fd_nnz(ctypes.byref(_grid(ns))))


def rhif_assemble_fd(ns, a_pix: torch.Tensor, b=0.0, stream=None):
    """Finite-difference matrix on the device: returns (rowptr int64, col int32, val float64)."""
    load()
    g = _grid(ns)
    N = 1
    for v in ns:
        N *= int(v)
    _need(a_pix, "a_pix", _npix(ns))
    if isinstance(b, torch.Tensor):
        _need(b, "b", N)
        _on_device(b=b)
    _on_device(a_pix=a_pix)
    nnz = int(_lib.rhif_fd_nnz(ctypes.byref(g)))
    dev = a_pix.device
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    a_pix = a_pix.contiguous().to(torch.float64)
    if isinstance(b, torch.Tensor):
        bn, bc = _ptr(b.contiguous().to(torch.float64)), 0.0
    else:
        bn, bc = None, float(b)
    _check(_lib.rhif_assemble_fd(ctypes.byref(g), _ptr(a_pix), bn, bc, _ptr(rowptr), _ptr(col),
                                 _ptr(val), _stream(stream)))
    return rowptr, col, val


class Factor:
    """A factor F ~= A owned by the library (free with :meth:`free`)."""

    def __init__(self, handle, ns, keep):
        self._h = handle
        self.ns = tuple(int(v) for v in ns)
        self.N = 1
        for v in self.ns:
            self.N *= v
        self._keep = keep

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def free(self):
        if self._h:
            _lib.rhif_free(self._h)
            self._h = None

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None,
              op: str = "solve") -> torch.Tensor:
        """op(F) x for x of shape (N,) or (nrhs, N): "solve" F^{-1} (Eq. 3.2),
        "matvec" F (Eq. 3.1), "half" G^{-1}, "half_t" G^{-T} (F = G G^T, Eq. 3.3)."""
        nrhs, ld = _cols(x, self.N)
        if out is not None:
            _need(out, "out", x.numel(), torch.float64)
            _on_device(out=out)
        y = torch.empty_like(x) if out is None else out
        code = {"solve": RHIF_SOLVE, "matvec": RHIF_MATVEC, "half": RHIF_HALF,
                "half_t": RHIF_HALF_T}[op]
        _check(_lib.rhif_apply(self._h, code, nrhs, _ptr(x), ld, _ptr(y), ld, _stream(stream)))
        return y

    def matvec(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        """F x (Eq. 3.1)."""
        return self.apply(x, stream=stream, op="matvec")

    def estimate_ea(self, x0: torch.Tensor, x1: torch.Tensor | None = None, maxit: int = 100,
                    rel: float = 1e-2, stream=None):
        """e_a = ||A - F||_2 / ||A||_2 by power iteration from the device vectors
        x0 (numerator) and x1 (denominator; default x0); returns (estimate, products)."""
        _need(x0, "x0", self.N, torch.float64)
        _on_device(x0=x0)
        if x1 is not None:
            _need(x1, "x1", self.N, torch.float64)
            _on_device(x1=x1)
        ea = ctypes.c_double()
        it = ctypes.c_int()
        _check(_lib.rhif_estimate_ea(self._h, _ptr(x0.contiguous()),
                                     _ptr(x1.contiguous()) if x1 is not None else None, int(maxit),
                                     float(rel), ctypes.byref(ea), ctypes.byref(it), _stream(stream)))
        return ea.value, it.value

    def apply_noalloc(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """F^{-1} x into the caller's ``out`` without any device allocation
        (library-owned static scratch; see rhif_apply_noalloc in rhif.h)."""
        nrhs, ld = _cols(x, self.N)
        _need(out, "out", x.numel(), torch.float64)
        _on_device(out=out)
        _check(_lib.rhif_apply_noalloc(self._h, nrhs, _ptr(x), ld, _ptr(out), ld, _stream(stream)))
        return out

    def spmv(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        nrhs, ld = _cols(x, self.N)
        y = torch.empty_like(x)
        _check(_lib.rhif_spmv(self._h, nrhs, _ptr(x), ld, _ptr(y), ld, _stream(stream)))
        return y

    def pcg(self, f: torch.Tensor, rtol=1e-10, maxit=1000, out=None, stream=None, check=True):
        """PCG with F^{-1}; returns (u, iters list, relres list)."""
        nrhs, ld = _cols(f, self.N)
        if out is not None:
            _need(out, "out", f.numel(), torch.float64)
            _on_device(out=out)
        u = torch.empty_like(f) if out is None else out
        it = (ctypes.c_int * nrhs)()
        rr = (ctypes.c_double * nrhs)()
        rc = _lib.rhif_pcg(self._h, nrhs, _ptr(f), ld, _ptr(u), ld, float(rtol), int(maxit), it, rr,
                           _stream(stream))
        if rc != 0 and (check or rc != -3):
            _check(rc)
        return u, list(it), list(rr)

    def estimate_es(self, x0: torch.Tensor, maxit: int = 100, rel: float = 1e-2, stream=None):
        """e_s = ||I - A F^{-1}||_2 by power iteration from the device vector x0;
        returns (estimate, number of M^T M products)."""
        _need(x0, "x0", self.N, torch.float64)
        _on_device(x0=x0)
        es = ctypes.c_double()
        it = ctypes.c_int()
        _check(_lib.rhif_estimate_es(self._h, _ptr(x0.contiguous()), int(maxit), float(rel),
                                     ctypes.byref(es), ctypes.byref(it), _stream(stream)))
        return es.value, it.value

    def stats(self) -> dict:
        st = Stats()
        _check(_lib.rhif_stats(self._h, ctypes.byref(st)))
        return {"levels": st.levels, "n": st.n, "root_size": st.root_size,
                "active": list(st.active)[:st.levels], "factor_bytes": st.factor_bytes,
                "flops": st.flops, "apply_bytes": st.apply_bytes, "precision": st.precision,
                "units": st.units, "factor_ms": st.factor_ms, "fp64_leaves": st.fp64_leaves,
                "unit_dofs": list(st.unit_dofs)[:st.levels],
                "skeletons": list(st.skeletons)[:st.levels]}

    def skeletons(self, level: int, phase: int = 0):
        """[(dofs in pivot order, rank)] for every unit of a level/phase."""
        cnt = ctypes.c_int()
        _check(_lib.rhif_skeletons(self._h, level, phase, ctypes.byref(cnt), None, None, None, 0))
        n = cnt.value
        sizes = (ctypes.c_int * max(n, 1))()
        ranks = (ctypes.c_int * max(n, 1))()
        _check(_lib.rhif_skeletons(self._h, level, phase, ctypes.byref(cnt), sizes, ranks, None, 0))
        tot = sum(sizes[i] for i in range(n))
        gids = (ctypes.c_int64 * max(tot, 1))()
        _check(_lib.rhif_skeletons(self._h, level, phase, ctypes.byref(cnt), sizes, ranks, gids, tot))
        out, pos = [], 0
        for i in range(n):
            out.append((list(gids[pos:pos + sizes[i]]), ranks[i]))
            pos += sizes[i]
        return out


def rhif_factor(csr, ns, leaf: int, tol: float, precision: str = "fp64", precondition=True,
                edge_skel_3d=False, stream=None, big_front=0, big_frame=0,
                skel_cluster=0, tensor_cores=0, leaf_fp64=0) -> Factor:
    """PHIF factorization of the CSR matrix ``csr = (rowptr, col, val)`` on grid ``ns``.
    ``big_front`` / ``big_frame`` / ``skel_cluster`` are the scheduling options of
    ``rhif_opts``; ``leaf_fp64`` the FP64 leaf fallback of FP32 factors."""
    load()
    A = _csr(csr, ns)
    o = _opts(precision, precondition, edge_skel_3d, big_front, big_frame, skel_cluster,
              tensor_cores, leaf_fp64)
    h = ctypes.c_void_p()
    _check(_lib.rhif_factor(ctypes.byref(A), ctypes.byref(_grid(ns)), int(leaf), float(tol),
                            ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    return Factor(h, ns, None)


class BatchFactor(Factor):
    """A merged factorization of several independent problems
    (rhif_factor_batch): one handle, the problems' DOFs numbered consecutively
    from ``dof_base[i]``; ``apply`` / ``spmv`` work on concatenated vectors of
    length ``N`` (the total), ``pcg_batch`` on one right-hand-side block per
    problem."""

    def __init__(self, handle, grids):
        super().__init__(handle, (1,), None)
        self.grids = [tuple(int(v) for v in g) for g in grids]
        cnt = ctypes.c_int()
        base = (ctypes.c_int64 * (len(grids) + 1))()
        _check(_lib.rhif_batch_info(self._h, ctypes.byref(cnt), base))
        self.dof_base = list(base)
        self.N = self.dof_base[-1]
        self.ns = (self.N,)

    def split(self, x: torch.Tensor):
        """Views of a concatenated vector (N,) or (nrhs, N), one per problem."""
        return [x[..., self.dof_base[i]:self.dof_base[i + 1]] for i in range(len(self.grids))]

    def pcg(self, f: torch.Tensor, rtol=1e-10, maxit=1000, out=None, stream=None, check=True):
        """PCG for every problem on concatenated vectors; iters / relres are
        lists of per-problem lists."""
        nrhs, ld = _cols(f, self.N)
        u = torch.empty_like(f) if out is None else out
        n = len(self.grids)
        it = (ctypes.c_int * (n * nrhs))()
        rr = (ctypes.c_double * (n * nrhs))()
        rc = _lib.rhif_pcg(self._h, nrhs, _ptr(f), ld, _ptr(u), ld, float(rtol), int(maxit), it, rr,
                           _stream(stream))
        if rc != 0 and (check or rc != -3):
            _check(rc)
        return u, [list(it[i * nrhs:(i + 1) * nrhs]) for i in range(n)], \
            [list(rr[i * nrhs:(i + 1) * nrhs]) for i in range(n)]

    def pcg_batch(self, fs, rtol=1e-10, maxit=1000, stream=None, check=True):
        """PCG with one right-hand-side block per problem: fs[i] of shape (N_i,)
        or (nrhs, N_i); returns (us, iters, relres) as per-problem lists."""
        n = len(self.grids)
        if len(fs) != n:
            raise ValueError("one right-hand-side block per problem")
        nrhs = 1 if fs[0].dim() == 1 else fs[0].shape[0]
        for i, f in enumerate(fs):
            _need(f, "f", nrhs * (self.dof_base[i + 1] - self.dof_base[i]), torch.float64)
            _on_device(f=f)
            assert f.is_contiguous(), "right-hand sides must be contiguous"
        us = [torch.empty_like(f) for f in fs]
        Fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fs])
        Up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
        it = (ctypes.c_int * (n * nrhs))()
        rr = (ctypes.c_double * (n * nrhs))()
        rc = _lib.rhif_pcg_batch(self._h, nrhs, Fp, Up, float(rtol), int(maxit), it, rr,
                                 _stream(stream))
        if rc != 0 and (check or rc != -3):
            _check(rc)
        return us, [list(it[i * nrhs:(i + 1) * nrhs]) for i in range(n)], \
            [list(rr[i * nrhs:(i + 1) * nrhs]) for i in range(n)]


def rhif_factor_batch(csrs, grids, leaf: int, tol: float, precision: str = "fp64",
                      precondition=True, edge_skel_3d=False, stream=None, **sched) -> BatchFactor:
    """One merged PHIF factorization of independent problems (one launch per
    level step across all of them); csrs[i] = (rowptr, col, val) on grid grids[i]."""
    load()
    n = len(csrs)
    A = (CSR * n)()
    G = (Grid * n)()
    for i, (csr, ns) in enumerate(zip(csrs, grids)):
        A[i] = _csr(csr, ns)
        G[i] = _grid(ns)
    o = _opts(precision, precondition, edge_skel_3d, **sched)
    h = ctypes.c_void_p()
    _check(_lib.rhif_factor_batch(n, A, G, int(leaf), float(tol), ctypes.byref(o), _stream(stream),
                                  ctypes.byref(h)))
    return BatchFactor(h, grids)


def rhif_autotune(csr, ns, leaf: int, tol: float, precision: str = "fp64", precondition=True,
                  edge_skel_3d=False, applies: int = 10, stream=None):
    """Scheduling options picked by the library's autotuner for this problem
    (see ``rhif_autotune`` in rhif.h): returns (dict of rhif_factor keyword
    arguments, cost in ms)."""
    load()
    A = _csr(csr, ns)
    o = _opts(precision, precondition, edge_skel_3d)
    best = Opts()
    ms = ctypes.c_double()
    _check(_lib.rhif_autotune(ctypes.byref(A), ctypes.byref(_grid(ns)), int(leaf), float(tol),
                              ctypes.byref(o), int(applies), _stream(stream), ctypes.byref(best),
                              ctypes.byref(ms)))
    kw = dict(precision=precision, precondition=precondition, edge_skel_3d=edge_skel_3d,
              big_front=best.big_front, big_frame=best.big_frame,
              skel_cluster=best.skel_cluster, tensor_cores=best.tensor_cores)
    return kw, ms.value


TC_KINDS = {"tf32x3": 0, "tf32": 1, "bf16": 2}


def rhif_tc_gemm_check(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, stream=None,
                       kind: str = "tf32x3"):
    """C -= A B^T on the tensor cores (operands: "tf32x3" split TF32, "tf32" or
    "bf16"); A (M, K), B (N, K), C (M, N) FP32 tensors given in column-major
    order, i.e. as the transposes of row-major tensors: pass
    A.t().contiguous().t() etc."""
    load()
    M, K = A.shape
    N = B.shape[0]
    lda = max(int(A.stride(1)), M) if K > 0 else M
    ldb = max(int(B.stride(1)), N) if K > 0 else N
    _check(_lib.rhif_tc_gemm_check(TC_KINDS[kind], int(M), int(N), int(K), _colptr(A), lda,
                                   _colptr(B), ldb,
                                   _colptr(C), max(int(C.stride(1)), M), _stream(stream)))
    return C


def rhif_plan_selfcheck(ns, leaf: int, keep: float = 0.5, seed: int = 1, edge_skel_3d=False) -> int:
    """Host-only check of the level plans of a grid (no GPU needed); returns
    the number of levels checked, raises RhifError on a violated invariant."""
    load()
    n = (ctypes.c_int * 3)(*[int(v) for v in ns], *([1] * (3 - len(ns))))
    levels = ctypes.c_int64(0)
    _check(_lib.rhif_plan_selfcheck(len(ns), n, int(leaf), float(keep), int(seed),
                                    int(bool(edge_skel_3d)), ctypes.byref(levels)))
    return int(levels.value)


def rhif_grad_logcoef(ns, a_pix: torch.Tensor, u: torch.Tensor, lam: torch.Tensor, stream=None):
    """dL/dlog a per pixel from the solution u and the adjoint lam (one right-hand side)."""
    load()
    _need(a_pix, "a_pix", _npix(ns), torch.float64)
    _need(u, "u", _ndof(ns), torch.float64)
    _need(lam, "lam", _ndof(ns), torch.float64)
    _on_device(a_pix=a_pix, u=u, lam=lam)
    grad = torch.empty_like(a_pix)
    _check(_lib.rhif_grad_logcoef(ctypes.byref(_grid(ns)), _ptr(a_pix), _ptr(u), _ptr(lam),
                                  _ptr(grad), _stream(stream)))
    return grad


def rhif_set_timing(on: bool):
    """CUDA-event timing of every library kernel launch (process-wide)."""
    load()
    _check(_lib.rhif_set_timing(1 if on else 0))


def rhif_reset_kernel_stats():
    load()
    _check(_lib.rhif_reset_kernel_stats())


def rhif_kernel_stats() -> dict:
    """{category: {launches, total_ms, flops, bytes}} since the last reset."""
    load()
    out = {}
    for i in range(_lib.rhif_kernel_stat_count()):
        st = KernelStat()
        _check(_lib.rhif_kernel_stats(i, ctypes.byref(st)))
        out[st.name.decode()] = {"launches": st.launches, "total_ms": st.total_ms,
                                 "flops": st.flops, "bytes": st.bytes}
    return out


def rhif_assemble_fd_log(ns, log_a_pix: torch.Tensor, b=0.0, stream=None):
    """Finite-difference matrix from the per-pixel log-coefficient; returns (csr, a_pix)."""
    load()
    g = _grid(ns)
    N = 1
    for v in ns:
        N *= int(v)
    _need(log_a_pix, "log_a_pix", _npix(ns))
    if isinstance(b, torch.Tensor):
        _need(b, "b", N)
        _on_device(b=b)
    _on_device(log_a_pix=log_a_pix)
    nnz = int(_lib.rhif_fd_nnz(ctypes.byref(g)))
    dev = log_a_pix.device
    log_a_pix = log_a_pix.contiguous().to(torch.float64)
    a_pix = torch.empty_like(log_a_pix)
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    if isinstance(b, torch.Tensor):
        bn, bc = _ptr(b.contiguous().to(torch.float64)), 0.0
    else:
        bn, bc = None, float(b)
    _check(_lib.rhif_assemble_fd_log(ctypes.byref(g), _ptr(log_a_pix), _ptr(a_pix), bn, bc,
                                     _ptr(rowptr), _ptr(col), _ptr(val), _stream(stream)))
    return (rowptr, col, val), a_pix


class RhifSolve(torch.autograd.Function):
    """u = A(log a)^{-1} f by PHIF-preconditioned CG, differentiable in log a and f.

    Forward: assemble A from exp(log a), factor it (PHIF, Sec. 3) and solve by
    PCG.  Backward: the adjoint lam = A^{-1} dL/du reuses the same factor (A is
    symmetric), dL/df = lam and dL/dlog a_p = -lam^T (dA/dlog a_p) u from the
    gradient kernel.  ``opts`` = dict(leaf, tol, precision, rtol, maxit).
    """

    @staticmethod
    def forward(ctx, log_a, f, ns, opts):
        o = dict(leaf=16, tol=1e-6, precision="fp64", rtol=1e-12, maxit=1000)
        o.update(opts or {})
        csr, a_pix = rhif_assemble_fd_log(ns, log_a.detach())
        F = rhif_factor(csr, ns, o["leaf"], o["tol"], precision=o["precision"])
        u, its, rr = F.pcg(f.detach().contiguous(), rtol=o["rtol"], maxit=o["maxit"])
        ctx.F, ctx.ns, ctx.o = F, tuple(ns), o
        ctx.save_for_backward(a_pix, u)
        ctx.iters = its
        return u

    @staticmethod
    def backward(ctx, g_u):
        a_pix, u = ctx.saved_tensors
        F = ctx.F
        lam, _, _ = F.pcg(g_u.contiguous(), rtol=ctx.o["rtol"], maxit=ctx.o["maxit"])
        grad_log_a = rhif_grad_logcoef(ctx.ns, a_pix, u, lam)
        F.free()
        ctx.F = None
        return grad_log_a, lam, None, None


def rhif_solve(log_a: torch.Tensor, f: torch.Tensor, ns, **opts) -> torch.Tensor:
    """Differentiable PHIF solve (see :class:`RhifSolve`)."""
    return RhifSolve.apply(log_a, f, tuple(ns), opts)


def _opts(precision="fp64", precondition=True, edge_skel_3d=False, big_front=0,
          big_frame=0, skel_cluster=0, tensor_cores=0, leaf_fp64=0) -> Opts:
    o = Opts()
    _lib.rhif_default_opts(ctypes.byref(o))
    o.precision = {"fp64": RHIF_FP64, "fp32": RHIF_MIXED_FP32, "mixed": RHIF_MIXED_FP32,
                   "tf32": 2, "bf16": 3}[precision]
    if isinstance(precondition, str):
        o.precondition = {"none": 0, "hif": 0, "block": 1, "phif": 1, "diag": 2}[precondition]
    else:
        o.precondition = 1 if precondition else 0
    o.edge_skel_3d = 1 if edge_skel_3d else 0
    o.big_front = int(big_front)
    o.big_frame = int(big_frame)
    o.skel_cluster = int(skel_cluster)
    o.tensor_cores = int(tensor_cores)
    o.leaf_fp64 = int(leaf_fp64)
    return o


def rhif_factor_batched(csrs, grids, leaf: int, tol: float, precision: str = "fp64",
                        precondition=True, streams=None):
    """Factor many independent problems concurrently (one worker per stream)."""
    load()
    n = len(csrs)
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(min(8, max(n, 1)))]
    A = (CSR * n)()
    G = (Grid * n)()
    for i, (csr, ns) in enumerate(zip(csrs, grids)):
        A[i] = _csr(csr, ns)
        G[i] = _grid(ns)
    S = (ctypes.c_void_p * len(streams))(*[s.cuda_stream for s in streams])
    out = (ctypes.c_void_p * n)()
    o = _opts(precision, precondition)
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    rc = _lib.rhif_factor_batched(n, A, G, int(leaf), float(tol), ctypes.byref(o), S, len(streams), out)
    facs = [Factor(ctypes.c_void_p(out[i]), grids[i], None) if out[i] else None for i in range(n)]
    for s in streams:
        cur.wait_stream(s)
    if rc != 0:
        for F in facs:
            if F is not None:
                F.free()
        _check(rc)
    return facs, streams


def rhif_pcg_batched(factors, fs, rtol=1e-10, maxit=1000, streams=None):
    """PCG for many factored problems at once; fs[i] is (nrhs, N_i).  Returns (us, iters, relres)."""
    load()
    n = len(factors)
    if len(fs) != n:
        raise ValueError("one right-hand-side block per factor")
    nrhs = 1 if fs[0].dim() == 1 else fs[0].shape[0]
    for F, f in zip(factors, fs):
        _need(f, "f", nrhs * F.N, torch.float64)
        _on_device(f=f)
        assert f.is_contiguous(), "right-hand sides must be contiguous"
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(min(8, max(n, 1)))]
    us = [torch.empty_like(f) for f in fs]
    H = (ctypes.c_void_p * n)(*[F._h.value if isinstance(F._h, ctypes.c_void_p) else F._h for F in factors])
    Fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fs])
    Up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
    it = (ctypes.c_int * (n * nrhs))()
    rr = (ctypes.c_double * (n * nrhs))()
    S = (ctypes.c_void_p * len(streams))(*[s.cuda_stream for s in streams])
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    rc = _lib.rhif_pcg_batched(n, H, nrhs, Fp, Up, float(rtol), int(maxit), it, rr, S, len(streams))
    for s in streams:
        cur.wait_stream(s)
    _check(rc)
    return us, [list(it[i * nrhs:(i + 1) * nrhs]) for i in range(n)], \
        [list(rr[i * nrhs:(i + 1) * nrhs]) for i in range(n)]
