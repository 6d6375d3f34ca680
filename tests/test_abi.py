"""The C ABI library loads without a GPU and exports every symbol the public
header declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdfcheck.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("SDF_")))


@pytest.fixture(scope="module")
def libpath():
    from paper_2309_12543_gb300 import build
    return build.build()


def test_header_declares_the_check_boundary():
    names = declared_functions()
    for n in ("sdf_build_grids", "check_trajectory", "sdf_ctx_create", "sdf_robot_create"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    import paper_2309_12543_gb300 as sdf
    assert sorted(sdf.EXPORTED) == declared_functions()


def test_binding_constants_match_header():
    import paper_2309_12543_gb300 as sdf
    text = open(HEADER).read()
    for name, val in re.findall(r"#define (SDF_\w+) \(?(-?\d+)\)?", text):
        if hasattr(sdf._native, name):
            assert getattr(sdf._native, name) == int(val), name


def test_fault_injection_counter_on_the_host(libpath):
    """The allocation-failure countdown is host state: armed, read back and
    disarmed without a GPU; a negative countdown is rejected."""
    import paper_2309_12543_gb300 as sdf
    count, nbytes, countdown = sdf.sdf_debug_alloc_live()
    assert count >= 0 and nbytes >= 0 and countdown == 0
    sdf.sdf_debug_fail_alloc(5)
    assert sdf.sdf_debug_alloc_live()[2] == 5
    sdf.sdf_debug_fail_alloc(0)
    assert sdf.sdf_debug_alloc_live()[2] == 0
    with pytest.raises(sdf.SdfError):
        sdf.sdf_debug_fail_alloc(-1)
