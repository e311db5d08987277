"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

from paper_2405_06997_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"WFPG_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for n in ("svo_build", "svo_accumulate", "bin_rays", "guide_build_pdf", "guide_sample",
              "guide_eval_pdf"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_is_empty_string_initially():
    lib = ctypes.CDLL(build.build())
    lib.wfpg_last_error.restype = ctypes.c_char_p
    assert lib.wfpg_last_error() == b""
