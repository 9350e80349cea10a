"""The C-ABI library builds, loads and exports every symbol that
include/geek.h declares (no GPU needed: no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "geek.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b((?:geek|silk)_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2106_10515_gb300 as pkg
    return pkg.build()


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T ((?:geek|silk)_\w+)$", out, flags=re.M))
    decl = declared_symbols()
    assert len(decl) >= 14
    missing = [s for s in decl if s not in exported]
    assert not missing, missing


def test_binding_lists_every_declared_symbol(libpath):
    from paper_2106_10515_gb300 import geek
    assert sorted(geek.EXPORTS) == declared_symbols()
    L = geek.lib()
    for s in geek.EXPORTS:
        assert hasattr(L, s)
    assert "sm_103a" in geek.version()


def test_library_built_for_sm103a_only(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True).stdout
    archs = set(re.findall(r"sm_(\d+a?)", out))
    assert archs == {"103a"}, archs


def test_context_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2106_10515_gb300 import geek
    import ctypes as C
    h = C.c_void_p()
    assert geek.lib().geek_ctx_create(0, C.byref(h)) != geek.OK
