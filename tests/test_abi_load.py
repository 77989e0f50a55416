"""The C-ABI library builds, loads without a GPU, and exports every symbol
declared in include/*.h (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b((?:hermite|hnn)_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1802_05246_b300 import build

    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    syms = declared_symbols()
    assert len(syms) >= 19
    for s in sorted(syms):
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b((?:hermite|hnn)_[a-z0-9_]+)\b", out))
    assert syms <= exported


def test_binding_lists_every_symbol(libpath):
    import paper_1802_05246_b300 as hb

    assert set(hb.EXPORTS) <= declared_symbols()
    hb.lib()  # loads and sets signatures without touching a GPU


def test_create_without_gpu_fails_cleanly(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1802_05246_b300 as hb

    with pytest.raises(hb.HermiteError):
        hb.Hermite(1, 3, 8, 1.0, 0.125, 0.1)


def test_argument_checks_need_no_gpu(libpath):
    import paper_1802_05246_b300 as hb

    L = hb.lib()
    h = ctypes.c_void_p()
    assert L.hermite_create(4, 3, 8, 1.0, 0.1, 0.05, 0, 0, ctypes.byref(h)) == -1
    assert L.hermite_create(1, 3, 8, 1.0, 0.1, 0.2, 0, 0, ctypes.byref(h)) == -1  # CFL > 1
    assert L.hermite_create(1, 0, 8, 1.0, 0.1, 0.05, 0, 0, ctypes.byref(h)) == -1  # m = 0 dissipative
    assert L.hermite_create(3, 4, 8, 1.0, 0.1, 0.05, 0, 0, ctypes.byref(h)) == -7
    assert b"compiled range" in L.hermite_last_error(None)
