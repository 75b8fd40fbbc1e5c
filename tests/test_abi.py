"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point that include/scff.h declares; argument errors are reported as
status codes, never as crashes."""
import ctypes
import os
import re

import pytest

from paper_2512_18010_b300 import scff

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(scff_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = scff.load()
    names = declared_functions()
    assert "scff_form_factor" in names and "scff_basis" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols():
    assert set(scff._SYMBOLS) <= set(declared_functions())


def test_null_arguments_return_status():
    lib = scff.load()
    assert lib.scff_create(None, 0, 0) == 1  # INVALID_ARG
    assert b"NULL" in lib.scff_last_error()
    assert lib.scff_form_factor(None, None, None, None, 0, 1.0, None, None, 0, None) == 1
    assert lib.scff_sync(None, None) == 1
    assert lib.scff_kernel_launches(None) == -1
    assert lib.scff_qgrid_size(None, None) == -1
    lib.scff_destroy(None)  # no-op


def test_library_has_no_oracle_dependency():
    # The product library and binding never reference the oracle.
    for fn in os.listdir(os.path.join(ROOT, "paper_2512_18010_b300")):
        if fn.endswith(".py"):
            src = open(os.path.join(ROOT, "paper_2512_18010_b300", fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
    csrc = os.path.join(ROOT, "paper_2512_18010_b300", "csrc")
    for fn in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, fn)).read().lower(), fn


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) == "", reason="device hidden")
def test_create_without_device_reports_error():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    with pytest.raises(scff.ScffError):
        scff.Context()
