"""The oracle and the CUDA path share no code.

The product package never imports, links or calls the oracle, and the oracle
never imports the product package; the only module both use is `synth`
(seeded input arrays).  Checked on the source text of both trees.
"""
from __future__ import annotations

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2507_04130_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                path = os.path.join(d, f)
                with open(path, encoding="utf-8") as fh:
                    yield path, fh.read()


def test_product_never_names_the_oracle():
    for path, text in _sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")):
        assert not re.search(r"\boracle\b", text, re.I), path


def test_oracle_never_imports_the_product():
    for path, text in _sources(ORACLE, (".py", ".c", ".h")):
        assert "paper_2507_04130_gb300" not in text, path
        assert "hipermotif.h" not in text and "libhipermotif" not in text, path


def test_synth_holds_no_matcher():
    with open(os.path.join(ROOT, "synth", "__init__.py"), encoding="utf-8") as fh:
        text = fh.read()
    assert "import oracle" not in text and "paper_2507_04130_gb300" not in text
    assert not re.search(r"def \w*(match|count_matches|enumerate)\w*\(", text)
