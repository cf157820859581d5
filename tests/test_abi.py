"""The C-ABI library loads without a GPU and exports every entry point the
header declares; the binding refuses to run without it."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "metade.h")).read()
    return sorted(set(re.findall(r"METADE_API\s+[\w\s\*]*?\b(metade_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("metade_create", "metade_inner_step", "metade_eval", "metade_outer_step"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import ctypes
    import paper_2502_10470_gb300 as M
    lib = ctypes.CDLL(M.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(M.EXPORTED) == declared_symbols()
    assert M.metade_strerror(M.METADE_EINVAL) == "invalid argument"
    # host-side argument checks answer before any device call
    assert M.metade_wait_check(2, 1)[0] == M.METADE_EINVAL
    assert M.metade_strerror(M.METADE_ETIMEOUT) == "device wait timed out"


def test_library_links_no_cpu_fallback():
    """The package has no compute path of its own: it only marshals arguments
    to libmetade.so and never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2502_10470_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "metade_oracle" not in text, f
