"""The C-ABI library: it builds for sm_103a, loads, and exports every entry point that
include/sacd.h declares (no compute calls: this runs without a GPU)."""

import os
import re
import subprocess

import pytest

from paper_2003_03572_gb300 import build as B
from paper_2003_03572_gb300 import sacd as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sacd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    if not os.path.exists(S.lib_path()):
        B.build()
    return S.lib_path()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("sacd_create", "sacd_mode_step", "sacd_iterate", "sacd_fit", "sacd_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(sacd_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = S.lib()
    for n in declared_functions():
        assert hasattr(L, n)


def test_build_targets_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_fails_loudly_without_gpu_or_library(tmp_path, monkeypatch):
    # with the library path pointing nowhere the binding raises instead of computing anything
    monkeypatch.setattr(S, "_LIB", None)
    monkeypatch.setattr(S, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        S.lib()
