"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, and its host-only entry points behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gbhe_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1207_1773_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as ex:  # the CUDA runtime must be loadable even without a GPU
        pytest.fail("libgbhegv.so does not load: %s" % ex)


def test_exports_every_declared_symbol(lib):
    decl = _declared()
    assert len(decl) >= 15
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1207_1773_gb300 import gbhegv
    assert set(gbhegv.exported_symbols()) == set(_declared())


def test_host_only_entry_points(lib):
    lib.gbhe_status_string.restype = ctypes.c_char_p
    assert lib.gbhe_status_string(0) == b"success"
    assert b"positive definite" in lib.gbhe_status_string(7)
    assert lib.gbhe_status_string(-103) == b"bounded device wait expired"
    v, t = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.gbhe_hb2st_sizes(100, 16, ctypes.byref(v), ctypes.byref(t)) == 0
    J = (100 - 1 + 15) // 16
    assert v.value == 100 * J * 16 and t.value == 100 * J
    assert lib.gbhe_hb2st_sizes(100, 0, None, None) == -2
    assert lib.gbhe_hb2st_sizes(-1, 8, None, None) == -1
    for n in (1, 100, 1000, 20000):
        nb = lib.gbhe_default_nb(n)
        assert 1 <= nb <= 128
    # argument checks happen before any device work
    assert lib.gbhe_potrf(None, 4, None, 4, None) == -1
    assert lib.gbhe_wait_selftest(None, None) == -1
    assert lib.gbhe_sync_status(None, None) == -1
    assert lib.gbhe_profile_enable(0) == 0
    lib.gbhe_launch_count.restype = ctypes.c_ulonglong
    assert lib.gbhe_launch_count() == 0


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1207_1773_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.c" not in src, f
