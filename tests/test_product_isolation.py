"""The product path is independent of the oracle and has no CPU fallback.

* no module of the package imports the oracle, and the oracle imports
  nothing from the package except the seeded input generators;
* the library's CUDA sources and the oracle's C++ sources include nothing
  from each other;
* the binding raises when libwfpg.so is missing instead of computing
  anything on the host.
"""
import ast
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2405_06997_gb300")


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mod = node.module or ""
            if node.level:  # relative import inside the package
                mod = "paper_2405_06997_gb300" + ("." + mod if mod else "")
            names.add(mod)
            names.update(f"{mod}.{a.name}" for a in node.names)
    return names


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(PKG, "*.py"))
    assert files
    for f in files:
        mods = imported_modules(f)
        assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (f, mods)


def test_oracle_uses_only_the_input_generators_from_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for m in imported_modules(f):
            if m.startswith("paper_2405_06997_gb300"):
                assert m in ("paper_2405_06997_gb300", "paper_2405_06997_gb300.inputs"), (f, m)


def test_native_sources_share_no_headers():
    cuda = glob.glob(os.path.join(PKG, "csrc", "*"))
    orc = glob.glob(os.path.join(ROOT, "oracle", "*.cpp")) + glob.glob(os.path.join(ROOT, "oracle", "*.h"))
    assert cuda and orc
    inc = re.compile(r'#\s*include\s*[<"]([^>"]+)[>"]')
    cuda_names = {os.path.basename(f) for f in cuda}
    orc_names = {os.path.basename(f) for f in orc}
    for f in orc:
        for h in inc.findall(open(f).read()):
            assert os.path.basename(h) not in cuda_names and "csrc" not in h and "wfpg.h" not in h, (f, h)
    for f in cuda:
        for h in inc.findall(open(f).read()):
            assert os.path.basename(h) not in orc_names and "oracle" not in h, (f, h)


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    from paper_2405_06997_gb300 import wfpg as W

    monkeypatch.setattr(W, "_lib", None)
    monkeypatch.setattr(W, "library_path", lambda: str(tmp_path / "missing" / "libwfpg.so"))
    with pytest.raises(RuntimeError, match="not built"):
        W.lib()
    with pytest.raises(RuntimeError, match="not built"):
        W.kernel_launches()


def test_host_tensors_are_refused_not_computed():
    """Host (CPU) tensors are refused with a TypeError before anything runs;
    no entry point computes on the host."""
    import numpy as np
    import torch

    from paper_2405_06997_gb300 import inputs
    from paper_2405_06997_gb300 import wfpg as W

    w = inputs.tiny_box(1)
    pdf, cr, cm = torch.zeros(4, 256), torch.zeros(4, 256), torch.zeros(4, 16)
    bins = torch.zeros(10, dtype=torch.int32)
    v3 = torch.zeros(10, 3)
    calls = [
        lambda: W.guide_sample(pdf, cr, cm, 16, bins, torch.zeros(10, 2)),
        lambda: W.guide_eval_pdf(pdf, 16, bins, v3),
        lambda: W.guide_sample_mix(pdf, cr, cm, 16, bins, v3, v3),
        lambda: W.guide_product_sums(pdf, 16),
        lambda: W.guide_product_sample(pdf, torch.zeros(4, 64), 16, bins, v3, v3),
        lambda: W.guide_product_eval(pdf, torch.zeros(4, 64), 16, bins, v3, v3),
        lambda: W.cast_rays(torch.from_numpy(w.scene.quads), torch.from_numpy(w.scene.spheres), v3, v3),
    ]
    for call in calls:
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()
    assert np.all(pdf.numpy() == 0)
