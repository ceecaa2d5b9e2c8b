"""The product path and the oracle share no code: nothing in the package or the CUDA
sources imports, includes or loads anything under oracle/, and the oracle does not
include the library's headers.  The product path has no CPU fallback: the binding
raises when liblbfs.so is missing."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2511_10257_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_package_does_not_use_the_oracle():
    for f in _files(PKG, (".py", ".cu", ".cuh", ".h")):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
        assert "lbfs_oracle" not in text and "liboracle" not in text, f


def test_oracle_does_not_use_the_library():
    for f in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2511_10257_gb300\b", text, re.M), f
        assert not re.search(r'#include\s+[<"][^>"]*lbfs\.h', text), f
        assert "liblbfs" not in text, f


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2511_10257_gb300 import lbfs
    with pytest.raises(OSError):
        lbfs.load(str(tmp_path / "missing" / "liblbfs.so"))
