"""The C-ABI library loads without a GPU and exports every function that
include/vm3dgs.h declares (no compute calls)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "include", "vm3dgs.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vm3dgs_[a-z0-9_]+)\s*\(", txt)))


def test_header_functions_exported():
    import paper_2506_19415_b300 as v
    lib = ctypes.CDLL(v.LIB_PATH)
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps every declared function
    assert set(names) <= set(v.EXPORTED)


def test_errors_are_reported_without_gpu():
    import paper_2506_19415_b300 as v
    import pytest
    import scenegen
    raw = scenegen.uniform_scene(n=100)
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=0))
    assert e.value.code == v.E_INVAL
    with pytest.raises(v.Vm3dgsError) as e:
        v.vm3dgs_build_pages(raw, v.BuildConfig(page_size=100, lod_levels=3, lod_fanout=8))
    assert e.value.code == v.E_INVAL and "divide" in str(e.value)
