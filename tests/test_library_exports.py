"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double)\s*\**\s*(\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    from paper_2304_09770_gb300 import LIB_PATH
    if not os.path.exists(LIB_PATH):
        from paper_2304_09770_gb300 import build_lib
        build_lib.build()
    return ctypes.CDLL(LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vem_assemble", "bddc_setup", "bddc_apply", "pcg_solve", "vem_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in _declared() if not hasattr(library, n)]
    assert not missing, missing
