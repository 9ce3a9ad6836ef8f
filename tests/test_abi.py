"""The C-ABI library builds, loads and exports every symbol include/tc.h declares.

No compute call is made here (no GPU needed): only symbol lookup and
tc_strerror, which touches no device state.
"""
import ctypes
import os
import re

import pytest

import paper_1308_2166_gb300 as tc
from paper_1308_2166_gb300 import build as tcbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tc_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    tcbuild.build()
    return tc.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(tc.EXPORTS)
    cdll = ctypes.CDLL(tc.LIB_PATH)
    for name in declared:
        assert hasattr(cdll, name), name


def test_strerror_without_gpu(lib):
    assert tc.tc_strerror(0) == "ok"
    for code in (tc.TC_ERR_INVAL, tc.TC_ERR_NOMEM, tc.TC_ERR_INPUT, tc.TC_ERR_CUDA,
                 tc.TC_ERR_TIMEOUT):
        assert tc.tc_strerror(code) not in ("ok", "unknown error")


def test_no_oracle_in_product_package():
    pkg = os.path.join(ROOT, "paper_1308_2166_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(tc, "_lib", None)
    with pytest.raises(RuntimeError):
        tc.load(str(tmp_path / "nope.so"))
