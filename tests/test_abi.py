"""The C ABI library loads on the CPU host and exports every entry point
declared in include/vct.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

from paper_2607_28872_b300 import build, vct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vct_status|void|const char \*)\s*\**\s*(\w+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(vct.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert vct.vct_strerror(vct.VCT_ERR_NOCONV) == "pressure solve did not converge"


def test_structs_match_header_sizes():
    # vct_params: 2 ints + 18 doubles + 4 ints + 6 doubles + 2 ints + 3 doubles
    assert ctypes.sizeof(vct.vct_params) == 8 + 18 * 8 + 16 + 48 + 8 + 24
    assert ctypes.sizeof(vct.vct_state) == 8 + 9 * 8
    assert ctypes.sizeof(vct.vct_stats) == 8 + 8 + 4 + 4 + 8 + 3 * 8
    assert ctypes.sizeof(vct.vct_bathymetry) == 5 * 8 + 8 + 4 * 8
