"""Host-side checks of the C ABI (no GPU needed, no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2102_01887_b300 import build as B
from paper_2102_01887_b300 import llama as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions() -> list[str]:
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(llama_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (llama_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "llama.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(llama_decision), offsetof(llama_decision, lat),
         offsetof(llama_decision, cost), offsetof(llama_decision, slack),
         offsetof(llama_decision, flags), sizeof(llama_opts));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    d = L.DECISION_DTYPE
    assert vals[:5] == [d.itemsize, d.fields["lat"][1], d.fields["cost"][1], d.fields["slack"][1],
                        d.fields["flags"][1]]
    assert vals[5] == ctypes.sizeof(L.llama_opts)


def test_constants_match_header():
    text = "".join(open(h).read() for h in HEADERS)
    for name, val in [("LLAMA_OK", L.OK), ("LLAMA_EINVAL", L.EINVAL), ("LLAMA_ENOMEM", L.ENOMEM),
                      ("LLAMA_ECUDA", L.ECUDA), ("LLAMA_ENOTREADY", L.ENOTREADY),
                      ("LLAMA_ETIMEOUT", L.ETIMEOUT), ("LLAMA_MODE_ALPHA", L.MODE_ALPHA),
                      ("LLAMA_FLAG_FEASIBLE", L.FLAG_FEASIBLE), ("LLAMA_FLAG_INVALID", L.FLAG_INVALID),
                      ("LLAMA_FLAG_TIMEOUT", L.FLAG_TIMEOUT), ("LLAMA_WAIT_LIMIT_DEFAULT", L.WAIT_LIMIT_DEFAULT),
                      ("LLAMA_MAX_HW", L.MAX_HW), ("LLAMA_MAX_CFG", L.MAX_CFG),
                      ("LLAMA_METHOD_STAIRCASE", L.METHOD_STAIRCASE), ("LLAMA_GEMM_RELU", L.GEMM_RELU),
                      ("LLAMA_DIRECT_DEFAULT", L.DIRECT_DEFAULT), ("LLAMA_DIRECT_LIMIT", L.DIRECT_LIMIT)]:
        m = re.search(rf"#define {name} \(?(-?\d+)( << (\d+))?\)?", text)
        assert m and int(m.group(1)) << int(m.group(3) or 0) == val, name


def test_create_rejects_bad_options_without_touching_a_gpu(lib):
    ctx = ctypes.c_void_p()
    for opts in [L.llama_opts(7, 3, 1, 1, 0, 0), L.llama_opts(0, 0, 1, 1, 0, 0),
                 L.llama_opts(0, 9, 1, 1, 0, 0), L.llama_opts(1, 3, 0, 1, 0, 0),
                 L.llama_opts(1, 3, 1, 70000, 0, 0)]:
        assert lib.llama_create(ctypes.byref(ctx), ctypes.byref(opts)) == L.EINVAL
    assert lib.llama_create(None, None) == L.EINVAL
    assert lib.llama_last_error(None) == b"null context"
    lib.llama_destroy(None)


def test_null_context_calls_fail_cleanly(lib):
    z = np.zeros(4, np.int64)
    assert lib.llama_set_queue(None, z.ctypes.data) == L.EINVAL
    assert lib.llama_schedule(None, 1, None, None, None, 0, None) == L.EINVAL
    assert lib.llama_reserve(None, 10) == L.EINVAL


def test_oracle_and_cuda_path_share_no_source():
    csrc = os.path.join(ROOT, "paper_2102_01887_b300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower().replace(
            "cpu oracle", ""), f
    orc = open(os.path.join(ROOT, "oracle", "llama_oracle.c")).read()
    assert "llama.h" not in orc and "csrc" not in orc
    for f in ("llama.py", "build.py", "workloads.py"):
        src = open(os.path.join(ROOT, "paper_2102_01887_b300", f)).read()
        assert "import oracle" not in src and "from oracle" not in src
