"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/fr.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_2306_06744_gb300 import build, fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(fr_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"fr_mesh_init", "fr_step", "fr_adapt", "fr_norms"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fr.EXPORTS) <= declared


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        return
    try:
        fr.Mesh({"dim": 2})
    except RuntimeError as e:
        assert "CUDA" in str(e)
    else:
        raise AssertionError("binding must refuse to run without a CUDA device")
