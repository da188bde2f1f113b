"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lspca.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1709_07175_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lspca_fit", "spca_fit", "lspca_project", "lspca_create", "lspca_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_1709_07175_gb300 import lspca
    assert set(_declared()) <= set(lspca.exported_symbols()) | set()
    lspca.load(libpath)
    assert lspca.lspca_strerror(0) == "ok"
    assert "invalid" in lspca.lspca_strerror(1)


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    from paper_1709_07175_gb300 import lspca
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lspca.LspcaError):
        lspca.lspca_create(0, 0)


def test_library_targets_sm_103a(libpath):
    # the build passes exactly one -gencode for sm_103a
    from paper_1709_07175_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_csr_binding_checks_array_types():
    """The CSR entry points take int64 row offsets, int32 column indices and
    FP32 values; the binding rejects other types before any library call, and
    passes null column / value pointers for an X without nonzeros."""
    import torch

    from paper_1709_07175_gb300 import lspca as L
    rp = torch.tensor([0, 1, 2], dtype=torch.int64)
    col = torch.tensor([0, 1], dtype=torch.int32)
    val = torch.tensor([1.0, 2.0], dtype=torch.float32)
    for bad in ((rp.int(), col, val), (rp, col.long(), val), (rp, col, val.double())):
        with pytest.raises(TypeError):
            L._csr_args(*bad)
    p_rp, p_col, p_val, m, nnz = L._csr_args(rp, col, val)
    assert (m, nnz) == (2, 2) and p_col is not None and p_val is not None
    empty = L._csr_args(torch.zeros(4, dtype=torch.int64), torch.zeros(0, dtype=torch.int32),
                        torch.zeros(0, dtype=torch.float32))
    assert empty[1] is None and empty[2] is None and empty[3:] == (3, 0)


def test_argument_checks_run_before_any_device_call(libpath):
    """Entry points reject bad arguments with LSPCA_ERR_INVALID before touching
    a device, so these calls are safe without a GPU."""
    from paper_1709_07175_gb300 import lspca as L
    lib = L.load(libpath)
    assert lib.lspca_sum_partials(None, None, 2, 10, None, None) == L.ERR_INVALID
    assert lib.lspca_wait_probe(None, 1000000, None, None) == L.ERR_INVALID
    assert lib.lspca_chain_noalloc(None, L.LSPCA_F32, 10, 10, 10, None, 64, None, None, None) == L.ERR_INVALID
