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


_C_PROGRAM = r"""
#include <stdio.h>
#include "gbhegv.h"
#include "gbhegv_probe.h"
int main(void) {
  int nm[2] = {500, 4000}, nb[2] = {32, 64}, out = 0, p[16], assign[3], ns[3] = {100, 300, 200}, rc;
  double fm[2] = {1.0, 1.0};
  unsigned W[64], M[4];
  size_t v2 = 0, t2 = 0, ws = 0;
  rc = gbhe_nb_rule_pick(2, nm, fm, nb, 3000, 300, &out);
  printf("%d %d\n", rc, out);
  rc = gbhe_crt_tables(p, W, M, NULL, NULL, NULL, NULL);
  printf("%d %d\n", rc, p[0]);
  rc = gbhe_batched_plan(2, 3, ns, assign);
  printf("%d %d %d %d\n", rc, assign[0], assign[1], assign[2]);
  rc = gbhe_hb2st_sizes(100, 16, &v2, &t2);
  printf("%d %zu %zu\n", rc, v2, t2);
  rc = gbhe_crt_workspace_size(128, 64, 32, 0, &ws);
  printf("%d %zu\n", rc, ws);
  printf("%d %s\n", gbhe_default_nb(10000), gbhe_status_string(GBHE_ETIMEOUT));
  return 0;
}
"""


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_is_plain_c_and_links(lib, tmp_path, compiler, std):
    """The public headers compile as C99 and as C++ (extern "C") without
    warnings, and a C program links libgbhegv.so and calls its host-only
    entry points."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(compiler + " not found")
    src = tmp_path / ("t.c" if compiler == "gcc" else "t.cpp")
    src.write_text(_C_PROGRAM)
    libdir = os.path.join(ROOT, "paper_1207_1773_gb300")
    exe = tmp_path / "t"
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L" + libdir, "-lgbhegv", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert out[0] == "0 64"
    assert out[1] == "16 256"
    assert out[2] == "0 1 0 1"                 # 300 -> worker 0, 200 -> worker 1, 100 -> worker 1
    J = (100 - 1 + 15) // 16
    assert out[3] == "0 %d %d" % (100 * J * 16, 100 * J)
    assert out[4].split()[0] == "0" and int(out[4].split()[1]) > 0
    assert out[5] == "64 bounded device wait expired"
