"""The C-ABI library builds, loads and exports every entry point that
include/ib.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ib.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(?:ib_status|void|const char|int32_t|int64_t|double|unsigned long long)\s*\**\s*(\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ib_init", "ib_interp", "ib_spread", "mg_solve", "ns_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1807_10504_gb300 as ib
    path = ib.build()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(ib.EXPORTS) == sorted(_declared())


def test_product_path_has_no_cpu_fallback(monkeypatch):
    import paper_1807_10504_gb300 as ib
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(ib.IBError):
        ib.Context(ib.Config(nx=16, ny=16, h=1 / 16), [0.5, 0.6, 0.5], [0.4, 0.5, 0.6], [0, 3])


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1807_10504_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower().replace(
                    "oracle", "oracle") or "import oracle" not in txt, f
                assert "import oracle" not in txt and "ib_oracle" not in txt, f
