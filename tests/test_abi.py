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


def test_product_path_and_oracle_are_separate():
    """The package (binding, batching, serving, CUDA sources) neither imports nor includes the oracle, and the
    oracle includes nothing of the CUDA path: the two share only the seeded input generator."""
    import ast
    pkg = os.path.join(ROOT, "paper_1804_03787_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            tree = ast.parse(open(os.path.join(pkg, f)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                assert not any(n.split(".")[0] == "oracle" for n in names), (f, names)
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^">]+)[">]', re.M)
    csrc = os.path.join(pkg, "csrc")
    for f in os.listdir(csrc):
        for h in inc.findall(open(os.path.join(csrc, f)).read()):
            assert "oracle" not in h, (f, h)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h")):
            for h in inc.findall(open(os.path.join(ROOT, "oracle", f)).read()):
                assert "gpm" not in h and "csrc" not in h and not h.endswith(".cuh"), (f, h)


def test_product_path_fails_loudly_without_a_gpu():
    """Importing the binding, batching and serving modules loads no oracle; without a CUDA device a context
    cannot be made (there is no CPU fallback)."""
    import subprocess
    import sys
    code = ("import sys, torch\n"
            "import paper_1804_03787_gb300.gpm as g, paper_1804_03787_gb300.batch, paper_1804_03787_gb300.serve\n"
            "assert 'oracle' not in sys.modules, 'oracle imported by the product path'\n"
            "if not torch.cuda.is_available():\n"
            "    try:\n"
            "        g.Context(g.default_params(), 64, 48)\n"
            "    except RuntimeError as e:\n"
            "        print('refused:', e)\n"
            "    else:\n"
            "        raise SystemExit('a context was made without a GPU')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
