"""The C-ABI library loads and exports every function include/nfftbl.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2502_07155_gb300 as nb
from paper_2502_07155_gb300 import build as nbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nfftbl.h")


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(nfftbl_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return nbuild.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nfftbl_plan", "nfftbl_set_nodes", "nfftbl_forward", "nfftbl_adjoint", "nfftbl_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly what the header declares
    assert sorted(nb.EXPORTED) == declared_functions()


def test_no_gpu_calls_fail_cleanly_on_host(libpath):
    """Argument validation runs before any device work."""
    lib = nb.lib()
    h = ctypes.c_void_p()
    M = (ctypes.c_int * 3)(256, 0, 0)
    assert lib.nfftbl_plan(ctypes.byref(h), 4, M, 2.0, 6, 0, None) == 1          # EINVAL: d
    assert b"d must be" in lib.nfftbl_plan_error()
    M1 = (ctypes.c_int * 3)(255, 0, 0)
    assert lib.nfftbl_plan(ctypes.byref(h), 1, M1, 2.0, 6, 0, None) == 1         # odd M
    assert lib.nfftbl_plan(ctypes.byref(h), 1, M, 2.0, 300, 0, None) == 1        # 2m >= L
    M3 = (ctypes.c_int * 3)(100, 0, 0)
    assert lib.nfftbl_plan(ctypes.byref(h), 1, M3, 1.1, 4, 0, None) == 3         # L = 110 = 2 5 11: not 2^a 3^b 5^c
    assert lib.nfftbl_plan(ctypes.byref(h), 1, M, 2.0, 13, 0, None) == 3         # m > 12
    assert lib.nfftbl_plan(None, 1, M, 2.0, 6, 0, None) == 1
    assert lib.nfftbl_destroy(None) == 0
    assert lib.nfftbl_set_nodes(None, 0, None) == 1
    assert lib.nfftbl_forward(None, None, None) == 1
    assert lib.nfftbl_last_error(None) == b"NULL plan"


def test_every_declaration_is_documented():
    """Each C-ABI declaration (or a group of adjacent ones) sits directly under
    a comment that states its meaning, layout, ownership and errors."""
    lines = open(HEADER).read().split("\n")
    undocumented = []
    for i, line in enumerate(lines):
        if re.match(r"^(nfftbl_status|const char\*|int64_t|int|size_t|void)\s+nfftbl_\w+\(", line):
            j = i - 1
            while j >= 0 and re.match(r"^(nfftbl_status|const char\*|int64_t|int|size_t|void)\s+nfftbl_\w+\(", lines[j]):
                j -= 1   # a group of declarations shares the comment above it
            while j >= 0 and lines[j].startswith(" ") and not lines[j].strip().endswith("*/"):
                j -= 1   # continuation lines of a multi-line declaration
            if j < 0 or not lines[j].rstrip().endswith("*/"):
                undocumented.append(line[:60])
    assert not undocumented, undocumented


def test_fig_5_1_frequency_grid():
    """v_s = -M/2 - m + s/S for s = 0 .. S (M + 2m) (Fig. 5.1)."""
    from paper_2502_07155_gb300.experiments import fig51_frequencies
    v = fig51_frequencies(20, 5, 32)
    assert v.size == 32 * 30 + 1
    assert v[0] == -15.0 and v[-1] == 15.0
    np.testing.assert_allclose(np.diff(v), 1 / 32, rtol=0, atol=1e-15)
