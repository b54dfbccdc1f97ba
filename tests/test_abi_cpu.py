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


def _header_text():
    return re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lens_sim.h")).read(), flags=re.S)


def _enum_block(text, name):
    m = re.search(r"typedef enum \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return {k: int(v) for k, v in re.findall(r"\b([A-Z][A-Z0-9_]*)\s*=\s*(-?\d+)", m.group(1))}


def _define(text, name):
    m = re.search(r"#define\s+" + name + r"\s+(-?\d+)\b", text)
    assert m, name
    return int(m.group(1))


def test_binding_constants_match_the_header():
    # the binding marshals by these numbers: a drift from the header would silently send the
    # wrong profile, light model or method to the library
    from paper_2606_01547_gb300 import lenssim, workloads
    text = _header_text()
    lens = {k[len("LENS_"):]: v for k, v in _enum_block(text, "lens_profile_type").items()}
    assert lens == lenssim.LENS_TYPES
    light = {k[len("LIGHT_"):]: v for k, v in _enum_block(text, "light_profile_type").items()}
    assert light == lenssim.LIGHT_TYPES
    status = _enum_block(text, "lens_status")
    assert {lenssim.STATUS_NAMES[v]: v for v in lenssim.STATUS_NAMES} == status
    assert _define(text, "LENS_PROFILE_PARAMS") == lenssim.PROFILE_PARAMS
    assert _define(text, "LENS_MAX_DEFLECTORS") == lenssim.MAX_DEFLECTORS
    assert {m: _define(text, "LENS_CONV_" + m.upper()) for m in lenssim.CONV_METHODS} == lenssim.CONV_METHODS
    assert _define(text, "LENS_CONV_FFT_MIN_K") == lenssim.CONV_FFT_MIN_K
    kern = open(os.path.join(ROOT, "paper_2606_01547_gb300", "csrc", "kernels.h")).read()
    assert int(re.search(r"kTraceVariants\s*=\s*(\d+)", kern).group(1)) == len(lenssim.TRACE_VARIANTS)
    assert _define(text, "LENS_TRACE_VARIANTS") == len(lenssim.TRACE_VARIANTS)
    assert int(re.search(r"kBatchForms\s*=\s*(\d+)", kern).group(1)) == len(lenssim.BATCH_FORMS)
    assert _define(text, "LENS_BATCH_FORMS") == len(lenssim.BATCH_FORMS)
    assert _define(text, "LENS_PIPE_RATES") == len(lenssim.PIPE_RATES)
    # every profile the library takes has a parameter layout in the input generators
    for name in list(lenssim.LENS_TYPES) + list(lenssim.LIGHT_TYPES):
        assert name in workloads.N_PARAMS, name
        assert workloads.N_PARAMS[name] <= lenssim.PROFILE_PARAMS
