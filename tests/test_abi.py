"""The C-ABI library builds, loads and exports every symbol include/tc.h declares.

No compute call is made here (no GPU needed): only symbol lookup and
tc_strerror, which touches no device state.
"""
import ctypes
import os
import re
import shutil
import subprocess

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


def _c_offsets(tmp_path, struct, fields):
    """offsetof() of each field and sizeof(struct) as the C compiler lays out
    the struct from include/tc.h."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "off.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tc.h"', 'int main(void) {']
    for f in fields:
        lines.append(f'  printf("%zu\\n", offsetof({struct}, {f}));')
    lines.append(f'  printf("%zu\\n", sizeof({struct}));')
    lines.append('  return 0; }')
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "off"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    return vals[:-1], vals[-1]


@pytest.mark.parametrize("struct,cls", [("tc_estimate_t", tc.tc_estimate_t),
                                        ("tc_profile_t", tc.tc_profile_t),
                                        ("tc_completion_t", tc.tc_completion_t),
                                        ("tc_server_config_t", tc.tc_server_config_t),
                                        ("tc_server_stats_t", tc.tc_server_stats_t)])
def test_struct_layout_matches_header(tmp_path, struct, cls):
    fields = [f for f, _ in cls._fields_]
    offs, size = _c_offsets(tmp_path, struct, fields)
    assert offs == [getattr(cls, f).offset for f in fields], struct
    assert size == ctypes.sizeof(cls), struct


def test_estimate_record_leads_with_problem_statement_fields():
    # the problem statement's result first: N (128-bit), r, |E|, the closed
    # count and tau_hat, then S and the batch count
    names = [f for f, _ in tc.tc_estimate_t._fields_]
    assert names[:6] == ["num_lo", "num_hi", "r", "m", "n_closed", "tau_hat"]
    assert tc.ESTIMATE_BYTES == 72


def test_completion_dtype_matches_struct():
    import numpy as np
    dt = tc._completion_dtype()
    assert dt.itemsize == ctypes.sizeof(tc.tc_completion_t)
    for name, _ in tc.tc_completion_t._fields_:
        assert dt.fields[name][1] == getattr(tc.tc_completion_t, name).offset, name
    assert np.dtype(dt.fields["tau_hat"][0]) == np.float64


def test_load_refuses_unreachable_tuples_on_the_host(lib):
    """tc_load checks a blob's tuples on the host before it creates a
    context, so these refusals need no GPU."""
    import numpy as np
    r, B = 4, 12
    empty = (1 << 64) - 1

    def blob(m, f1, f2, chi, fl):
        hdr = np.zeros(16, dtype=np.uint64)
        hdr[:11] = [0x3145544154534354, 1, r, 7, 0, B, m, 1 if m else 0, 0, 0, 0]
        return (hdr.tobytes() + np.array(f1, dtype=np.uint64).tobytes()
                + np.array(f2, dtype=np.uint64).tobytes()
                + np.array(chi, dtype=np.uint64).tobytes()
                + np.array(fl, dtype=np.uint32).tobytes())

    e = (1 << 32) | 2
    bad = [
        blob(0, [e, empty, empty, empty], [empty] * 4, [0] * 4, [0] * 4),   # edge before |E| > 0
        blob(10, [empty, e, e, e], [empty] * 4, [0] * 4, [0] * 4),          # empty f1 after
        blob(10, [(1 << 32) | (1 << B)] + [e] * 3, [empty] * 4, [0] * 4, [0] * 4),
        blob(10, [e] * 4, [(3 << 32) | 4] + [empty] * 3, [1, 0, 0, 0], [0] * 4),
        blob(10, [e] * 4, [empty] * 4, [2, 0, 0, 0], [0] * 4),
    ]
    for b in bad:
        h = ctypes.c_void_p()
        assert lib.tc_load(b, len(b), 4096, ctypes.byref(h)) == tc.TC_ERR_INVAL
        assert not h.value
