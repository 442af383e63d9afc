"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function
that include/mdot.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

from paper_2307_08507_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(mdot_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdot_solve", "mdot_dual_eval", "mdot_round", "mdot_create", "mdot_destroy"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_is_not_linked_into_the_product():
    """The product library and binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2307_08507_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "oracle.h" not in text, fn
