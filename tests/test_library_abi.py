"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ccmc.h declares (no GPU needed: nothing is computed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ccmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ccmc_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ccmc_init", "ccmc_step", "ccmc_energy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_1807_03749_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1807_03749_gb300.ccmc import EXPORTS

    assert sorted(EXPORTS) == _declared()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1807_03749_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "ccmc_oracle" not in text, f
