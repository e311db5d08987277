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


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the C layout (size and offset of
    every field) that include/wfpg.h gives."""
    import subprocess

    from paper_2405_06997_gb300 import wfpg as W

    structs = {"wfpg_scene": W.Scene, "wfpg_bin_params": W.BinParams, "wfpg_guide_params": W.GuideParams,
               "wfpg_camera": W.Camera, "wfpg_frame_params": W.FrameParams, "wfpg_frame_stats": W.FrameStats,
               "wfpg_learned_params": W.LearnedParams, "wfpg_adam_params": W.AdamParams,
               "wfpg_svo_info": W.SvoInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wfpg.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.split("\n") if line)
    for cname, cls in structs.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)
