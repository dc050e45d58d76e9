"""The C-ABI library builds for sm_103a, loads, and exports every symbol
include/gpm.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpm_[a-z_]+)\s*\(", src)) - {"gpm_alloc_fn", "gpm_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1804_03787_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_same_symbols():
    from paper_1804_03787_gb300 import gpm
    assert sorted(gpm.EXPORTED) == _declared()


def test_struct_layouts_match_header(lib):
    """Sizes of the ctypes mirrors agree with the C structs (x86-64 and aarch64 LP64)."""
    from paper_1804_03787_gb300 import gpm
    # 18 ints, 9 floats, census, the 8-byte seed, interp and tail padding to the seed's alignment
    assert ctypes.sizeof(gpm.Params) == 4 * (2 + 8 + 8) + 4 * 9 + 4 + 8 + 4 + 4
    assert gpm.Params.seed.offset == 112 and gpm.Params.interp.offset == 120
    assert ctypes.sizeof(gpm.Limits) == 24
    assert ctypes.sizeof(gpm.Pair) == 40


def test_host_only_calls_without_gpu(lib):
    """Parameter defaults and the memory estimate need no device."""
    from paper_1804_03787_gb300 import gpm
    L = gpm.load(build=False)
    p = gpm.Params()
    L.gpm_default_params(ctypes.byref(p))
    assert p.patch_radius == 3 and p.num_scales == 3 and list(p.cell_size)[:3] == [32, 16, 8]
    lim = gpm.Limits(1024, 436, 1, 0, 0)
    p.patch_radius = 4
    p.num_scales = 4
    for i, s in enumerate((64, 32, 16, 8)):
        p.cell_size[i] = s
    nb = L.gpm_required_bytes(ctypes.byref(p), ctypes.byref(lim))
    assert 50e6 < nb < 400e6
    assert L.gpm_status_string(1) == b"GPM_EINVAL"
    h = ctypes.c_void_p()
    bad = gpm.Limits(0, 0, 0, 0, 0)
    assert L.gpm_create(ctypes.byref(p), ctypes.byref(bad), gpm.ALLOC_FN(0), gpm.FREE_FN(0), None, None,
                        ctypes.byref(h)) == gpm.GPM_EINVAL
    p.cell_size[0] = 7
    assert L.gpm_create(ctypes.byref(p), ctypes.byref(lim), gpm.ALLOC_FN(0), gpm.FREE_FN(0), None, None,
                        ctypes.byref(h)) == gpm.GPM_EINVAL
