"""The C-ABI library builds, loads on the CPU host and exports every entry
point that include/*.h declares (no compute calls: no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*(?:\s+|\s*\*+\s*)([a-z_][a-z_0-9]*)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2201_05413_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fem_assemble", "fem_lift_rhs", "csr_to_sell", "pcg_solve", "pcg_solve_batched",
                     "fem_system_destroy", "sell_destroy", "gbpcg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import paper_2201_05413_gb300 as P
    L = P.load()
    assert b"sm_103a" in L.gbpcg_version()


def test_binding_marshals_every_declared_symbol():
    from paper_2201_05413_gb300 import gbpcg
    missing = [n for n in declared_functions() if n not in gbpcg._SIGS]
    assert not missing, missing


def test_product_package_never_imports_oracle():
    """The product path cannot route through the oracle (no import, no load)."""
    pkg = os.path.join(ROOT, "paper_2201_05413_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            txt = open(path).read()
            assert "import oracle" not in txt and "from oracle" not in txt, path
            assert "liboracle" not in txt and "orc_" not in txt, path
