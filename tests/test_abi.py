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
    return sorted(set(re.findall(r"\b(gpm_[a-z0-9_]+)\s*\(", src)) - {"gpm_alloc_fn", "gpm_free_fn"})


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
    # 18 ints, 9 floats, census, the 8-byte seed, interp and the sweep launch shape (no tail padding)
    assert ctypes.sizeof(gpm.Params) == 4 * (2 + 8 + 8) + 4 * 9 + 4 + 8 + 4 + 4
    assert gpm.Params.seed.offset == 112 and gpm.Params.interp.offset == 120
    assert gpm.Params.sweep_blocks_per_sm.offset == 124
    assert ctypes.sizeof(gpm.Limits) == 24
    assert ctypes.sizeof(gpm.Pair) == 40
    assert gpm.Pair.pair_id.offset == 32 and gpm.Pair.dtype.offset == 36  # per-pair frame dtype (gpm_dtype)


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


def _bench_params(gpm):
    p = gpm.Params()
    gpm.load(build=False).gpm_default_params(ctypes.byref(p))
    p.patch_radius = 4
    p.num_scales = 4
    for i, s in enumerate((64, 32, 16, 8)):
        p.cell_size[i] = s
    return p


def test_create_over_budget_is_busy_before_any_allocation(lib):
    """GPM_EBUSY: a budget below gpm_required_bytes refuses the context before the allocator is called."""
    from paper_1804_03787_gb300 import gpm
    L = gpm.load(build=False)
    p = _bench_params(gpm)
    calls = []
    alloc = gpm.ALLOC_FN(lambda user, nb, st: calls.append(nb) or 0)
    free = gpm.FREE_FN(lambda user, ptr, st: None)
    need = L.gpm_required_bytes(ctypes.byref(p), ctypes.byref(gpm.Limits(1024, 436, 2, 0, 0)))
    h = ctypes.c_void_p(1)
    lim = gpm.Limits(1024, 436, 2, 0, need - 1)
    assert L.gpm_create(ctypes.byref(p), ctypes.byref(lim), alloc, free, None, None, ctypes.byref(h)) == gpm.GPM_EBUSY
    assert not h.value and calls == []


def test_create_with_failing_allocator_is_enomem_and_frees_what_it_took(lib):
    """GPM_ENOMEM: the allocator callback returns NULL for the third slot; the two blocks it gave are freed
    through the free callback, and the caller gets no context."""
    from paper_1804_03787_gb300 import gpm
    L = gpm.load(build=False)
    p = _bench_params(gpm)
    given, freed = [], []

    def _alloc(user, nb, st):
        if len(given) == 2:
            return 0
        given.append(0x100000 * (len(given) + 1))
        return given[-1]

    alloc = gpm.ALLOC_FN(_alloc)
    free = gpm.FREE_FN(lambda user, ptr, st: freed.append(ptr))
    h = ctypes.c_void_p(1)
    lim = gpm.Limits(256, 192, 4, 0, 0)
    assert L.gpm_create(ctypes.byref(p), ctypes.byref(lim), alloc, free, None, None, ctypes.byref(h)) == gpm.GPM_ENOMEM
    assert not h.value
    assert sorted(freed) == sorted(given) and len(given) == 2


def test_create_without_a_device_is_ecuda():
    """GPM_ECUDA: on a host without a CUDA device a context cannot be made, even when the allocator callback
    succeeds (its blocks, one per pair, are handed back)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1804_03787_gb300 import gpm, build_lib
    build_lib.build()
    L = gpm.load(build=False)
    p = _bench_params(gpm)
    given, freed = [], []
    alloc = gpm.ALLOC_FN(lambda user, nb, st: given.append(0x200000 * (len(given) + 1)) or given[-1])
    free = gpm.FREE_FN(lambda user, ptr, st: freed.append(ptr))
    h = ctypes.c_void_p(1)
    lim = gpm.Limits(256, 192, 2, 0, 0)
    assert L.gpm_create(ctypes.byref(p), ctypes.byref(lim), alloc, free, None, None, ctypes.byref(h)) == gpm.GPM_ECUDA
    assert not h.value and sorted(freed) == sorted(given) and len(given) == 2


def test_every_status_code_has_a_name(lib):
    """The status codes the header lists, and only those, have names; GPM_OK and GPM_EINTERNAL are reached by the
    GPU tests (test_gpu_edges.py: the consistency flag), the others above."""
    from paper_1804_03787_gb300 import gpm
    L = gpm.load(build=False)
    src = open(os.path.join(ROOT, "include", "gpm.h")).read()
    codes = dict((m, int(v)) for m, v in re.findall(r"\b(GPM_E[A-Z]+|GPM_OK)\s*=\s*(\d+)", src))
    assert codes == {"GPM_OK": 0, "GPM_EINVAL": 1, "GPM_ENOMEM": 2, "GPM_ECUDA": 3, "GPM_EBUSY": 5,
                     "GPM_EINTERNAL": 6}
    for name, v in codes.items():
        assert L.gpm_status_string(v).decode() == name
        assert getattr(gpm, name) == v
    assert L.gpm_status_string(4) == b"unknown"
    # calls on a NULL context are refused without a device
    assert L.gpm_sync(None) == gpm.GPM_EINVAL and L.gpm_fit_planes(None, 1, 1) == gpm.GPM_EINVAL
