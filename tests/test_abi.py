"""The C-ABI library builds, loads and exports every symbol the header declares
(no compute: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "halosketch.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sketch_create", "sketch_update", "sketch_query", "topk_extract", "sketch_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1711_00975_gb300 import halosketch
    path = halosketch.lib()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_calls_fail_cleanly_without_a_device():
    # on a machine without a GPU the library reports an error instead of aborting
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1711_00975_gb300 import halosketch as hsk
    h = ctypes.c_void_p()
    p = hsk.make_params(5, 16, 100.0, 0.1, 1, 2)
    st = hsk.lib().sketch_create(ctypes.byref(p), 0, ctypes.byref(h))
    assert st != hsk.HS_OK and hsk.hs_last_error()
    assert hsk.lib().sketch_update(None, None, 5, 1.0) == hsk.HS_ERR_ARG


def test_argument_checks_need_no_device():
    from paper_1711_00975_gb300 import halosketch as hsk
    L = hsk.lib()
    h = ctypes.c_void_p()
    for bad in (hsk.make_params(0, 16, 100.0, 0.1), hsk.make_params(33, 16, 100.0, 0.1),
                hsk.make_params(5, 0, 100.0, 0.1), hsk.make_params(5, 31, 100.0, 0.1),
                hsk.make_params(5, 16, -1.0, 0.1), hsk.make_params(5, 16, 1e9, 1e-3),
                hsk.make_params(5, 16, 100.0, 0.1, flags=32),
                hsk.make_params(5, 16, 100.0, 0.1, flags=hsk.HS_FLAG_SEARCH_SCAN | hsk.HS_FLAG_SEARCH_DIRECTORY),
                hsk.make_params(5, 16, 100.0, 0.1, flags=hsk.HS_FLAG_UPDATE_DIRECT | hsk.HS_FLAG_UPDATE_BINNED)):
        assert L.sketch_create(ctypes.byref(bad), 0, ctypes.byref(h)) == hsk.HS_ERR_ARG
    assert L.sketch_create(None, 0, ctypes.byref(h)) == hsk.HS_ERR_ARG
    n = ctypes.c_uint32()
    assert L.topk_extract(None, 5, None, None, ctypes.byref(n)) == hsk.HS_ERR_ARG
    assert L.sketch_query(None, None, 3, None) == hsk.HS_ERR_ARG


def test_oracle_and_library_share_no_code():
    # neither side includes, imports or links the other
    lib_dir = os.path.join(ROOT, "paper_1711_00975_gb300")
    for dirpath, _, files in os.walk(lib_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", txt).lower(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1711_00975_gb300" not in txt and "hs_device" not in txt, f
