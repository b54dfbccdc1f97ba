"""CPU checks of the boundary: the library builds, loads and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(lens_[a-z_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("lens_sim_create", "lens_sim_image", "lens_sim_grad", "lens_serve_submit", "lens_serve_wait"):
        assert name in d


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2606_01547_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lens_[a-z_]+)", out))
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_without_gpu():
    pytest.importorskip("torch")
    from paper_2606_01547_gb300 import lenssim
    L = lenssim.lib()
    for name in lenssim.EXPORTED:
        assert hasattr(L, name)
    assert set(lenssim.EXPORTED) == _declared()
