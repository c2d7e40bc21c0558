"""The C-ABI library builds, loads and exports every entry point of include/qs.h (CPU only).

No compute call is made here: there is no GPU on this side.
"""
import ctypes
import os
import re

import pytest

from paper_1412_2293_gb300 import build, qs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ["qs_create", "qs_apply_gate", "qs_apply_noisy_gate", "qs_apply_kraus",
                     "qs_truncate_rank", "qs_fidelity", "qs_trace", "qs_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(qs._SIGS)


def test_binding_loads_without_a_device(libpath):
    L = qs.lib()
    assert qs.qs_version().startswith("paper_1412_2293_gb300")
    assert L is qs.lib()


def test_no_device_means_an_error_not_a_fallback(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(qs.QSError) as ei:
        qs.qs_create(4, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
    assert ei.value.status == qs.QS_ERR_CUDA


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1412_2293_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
