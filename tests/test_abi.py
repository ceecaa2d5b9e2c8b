"""The C ABI library builds, loads without a GPU and exports every function that
include/lbfs.h declares; the binding's structs match the header's layout."""
import ctypes as ct
import os
import re
import subprocess

import pytest

from paper_2511_10257_gb300 import build as B
from paper_2511_10257_gb300 import lbfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbfs_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbfs_create", "lbfs_set_case", "lbfs_step", "lbfs_fields", "lbfs_destroy",
                     "lbfs_last_error", "lbfs_set_fields"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ct.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, printed by a C program compiled with gcc"""
    body = "".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbfs.h"\n'
                    f'int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("struct,cls", [("lbfs_case_desc", "CaseDesc"), ("lbfs_case_stats", "CaseStats"),
                                        ("lbfs_config", "Config")])
def test_struct_layouts_match_header(struct, cls, tmp_path):
    C = getattr(lbfs, cls)
    names = [n for n, _ in C._fields_]
    size, offs = _c_layout(struct, names, tmp_path)
    assert ct.sizeof(C) == size
    assert [getattr(C, n).offset for n in names] == offs


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(OSError):
        lbfs._lib = None
        lbfs.load(str(tmp_path / "missing.so"))
    lbfs._lib = None
