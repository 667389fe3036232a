"""The C-ABI library loads and exports every entry point include/ara.h declares
(CPU only: no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ara.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^ARA_API[^;]*?\b(ara_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import importlib.util
    path = os.path.join(ROOT, "paper_1412_4556_b300", "build.py")
    spec = importlib.util.spec_from_file_location("ara_engine_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def test_header_declares_the_paper_boundary():
    names = declared_symbols()
    for n in ("ara_load_yet", "ara_load_elts", "ara_define_layer", "ara_layer_ylt", "ara_pml_tvar"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_binding_wraps_every_symbol_under_its_own_name(lib_path):
    from paper_1412_4556_b300 import _native
    for n in declared_symbols():
        assert n in _native.PROTOTYPES, n
        assert callable(getattr(_native, n)), n


def test_status_strings(lib_path):
    from paper_1412_4556_b300 import _native
    for code, name in _native.STATUS_NAMES.items():
        assert _native.ara_status_string(code) == name
    assert _native.ara_status_string(-99) == "ARA_E_UNKNOWN"


def test_create_without_gpu_reports_status_not_crash(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1412_4556_b300 import _native
    with pytest.raises(_native.AraError) as ei:
        _native.ara_create(0)
    assert ei.value.name == "ARA_E_CUDA"
    assert "device" in _native.ara_last_error(None)


def test_oracle_and_engine_share_no_code():
    """The oracle imports nothing from the engine and vice versa."""
    eng = os.path.join(ROOT, "paper_1412_4556_b300")
    orc = os.path.join(ROOT, "oracle")
    for d, other in ((eng, "oracle"), (orc, "paper_1412_4556_b300")):
        for dirpath, _, files in os.walk(d):
            for f in files:
                if f.endswith((".py", ".c", ".cu", ".cuh", ".h")):
                    src = open(os.path.join(dirpath, f)).read()
                    assert not re.search(rf"\b(import|from)\s+{other}\b", src), (f, other)
                    assert f'#include "{other}' not in src
