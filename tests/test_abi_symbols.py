"""The C-ABI library builds for sm_103a and exports every function that
include/rhif.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(rhif_\w+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["rhif_factor", "rhif_apply", "rhif_pcg", "rhif_free", "rhif_assemble_fd",
                 "rhif_grad_logcoef", "rhif_stats", "rhif_skeletons"]:
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1808_01364_gb300 import build
    if not build.up_to_date():
        build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_export():
    import paper_1808_01364_gb300 as rhif
    assert sorted(rhif.EXPORTS) == _declared()


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: when the CUDA library cannot be built, loading raises."""
    import paper_1808_01364_gb300 as rhif
    from paper_1808_01364_gb300 import build

    def no_nvcc(*a, **k):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")

    monkeypatch.setattr(rhif, "_lib", None)
    monkeypatch.setattr(build, "up_to_date", lambda: False)
    monkeypatch.setattr(build, "build", no_nvcc)
    with pytest.raises(RuntimeError, match="cannot be built"):
        rhif.load()
    with pytest.raises(RuntimeError, match="cannot be built"):
        rhif.rhif_fd_nnz((3, 3))
